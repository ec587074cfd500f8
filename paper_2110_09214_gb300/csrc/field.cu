// Field at points: BEM cell field (Eqs. (BEM3), (BEM2)) + all-pairs Coulomb
// field of point charges (Eq. (nbody)), the step's fused field, and the batch
// of chambers' field.
//
// Charges.  When the targets are the charges themselves (every step) the
// symmetric kernel evaluates each unordered pair once and applies the
// reaction to the other charge: tiles of 1024 charges paired cyclically,
// persistent blocks taking work units from a counter, sources rotated around
// the warp with their reaction sums, partial sums in slots of their own folded
// per charge in a fixed order (deterministic).  It runs on a copy of the
// charges ordered by charge value so that k_C q factors out of most tile
// pairs.  Separate targets and sources use the one-sided kernel: FT_TPT
// targets per thread as f32x2 packs, sources staged through shared memory as
// duplicated pairs, compensated (TwoSum) folds of every tile.
//
// Cells.  Targets are ordered along a 64^3 Morton grid (stable radix sort) and
// cut into blocks of <= 512; per block, cells near its box get the FP64
// closed form (targets within h) and a 112- or 28-point rule, the others one
// of the quadrature tiers of field_common.cuh (TIER_*_H2, far_point),
// emitted as point sources into the same packed loop as the charges.
#include "obem_internal.cuh"
#include "field_common.cuh"

#define FT_THREADS 128
#ifndef FT_TPT
#define FT_TPT 4                    // targets per thread (even)
#endif
#ifndef FT_MINB
#define FT_MINB 6                   // resident blocks per SM the register budget is cut for
#endif
#ifndef FT_UNROLL
#define FT_UNROLL 4                 // source-loop unrolling of the all-pairs kernel
#endif
#define FT_PRAGMA(x) _Pragma(#x)
#define FT_UNROLL_BY(n) FT_PRAGMA(unroll n)
#define FT_BLOCK_TARGETS (FT_THREADS * FT_TPT)
#define FT_SRC_TILE 256
#define FT_PAN_TILE 64

// Far-cell tiers (TIER_*_H2) and their rules (far_point): field_common.cuh.






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

// Blocks of the cell kernels: the targets of one super-bin (4 x 4 x 4 bins,
// contiguous in the sorted order) are cut into blocks of at most CT_BLOCK_N,
// so a block never spans distant bins.  One block of 1024 threads; reads the
// scanned histogram (bin start offsets) before the scatter advances it.
#define CT_BLOCK_N 512
__global__ void block_list_kernel(const int32_t *start, int nt_host, const int32_t *nt_dev, int2 *blocks,
                                  int32_t *nblocks)
{
    __shared__ int32_t part[1024];
    const int nt = nt_dev ? *nt_dev : nt_host;
    constexpr int PER = OBEM_NSUPER >= 1024 ? OBEM_NSUPER / 1024 : 1;
    const int per = OBEM_NSUPER >= 1024 ? PER : (threadIdx.x < OBEM_NSUPER ? 1 : 0);
    int cnt[PER];
    int32_t s = 0;
    for (int q = 0; q < per; ++q) {
        const int sb = threadIdx.x * per + q;
        const int a = start[sb << OBEM_SUPER_SHIFT];
        const int b = (sb + 1 < OBEM_NSUPER) ? start[(sb + 1) << OBEM_SUPER_SHIFT] : nt;
        cnt[q] = b - a;
        s += (b - a + CT_BLOCK_N - 1) / CT_BLOCK_N;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t o = part[threadIdx.x] - s;
    for (int q = 0; q < per; ++q) {
        const int sb = threadIdx.x * per + q;
        const int a = start[sb << OBEM_SUPER_SHIFT];
        for (int k = 0; k < cnt[q]; k += CT_BLOCK_N) blocks[o++] = make_int2(a + k, min(CT_BLOCK_N, cnt[q] - k));
    }
    if (threadIdx.x == 1023) nblocks[0] = part[1023];
}

// Target order of the cell kernels: a stable LSD radix sort of the bin codes
// (three passes of 6-bit digits over the 18-bit Morton code), so that each
// bin's targets keep their index order.  The order, hence every block's
// membership and every sum, is the same on every run (an atomic scatter would
// order each bin by the race).
#define RS_RADIX 64
#define RS_BLOCK 1024
int obem_binsort_blocks(int capacity) { return (capacity + RS_BLOCK - 1) / RS_BLOCK; }

// digit counts of each block of RS_BLOCK keys: rh[digit * nblk + block]
__global__ void rs_hist_kernel(const uint32_t *key, int nt, const int32_t *nt_dev, int shift, int nblk, int32_t *rh)
{
    __shared__ int32_t h[RS_RADIX];
    const int n = nt_dev ? *nt_dev : nt;
    if (threadIdx.x < RS_RADIX) h[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * RS_BLOCK + threadIdx.x;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & (RS_RADIX - 1)], 1);
    __syncthreads();
    if (threadIdx.x < RS_RADIX) rh[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of m counts in place (one block of 1024 threads)
__global__ void rs_scan_kernel(int32_t *a, int m)
{
    __shared__ int32_t part[1024];
    const int per = (m + 1023) / 1024, q0 = threadIdx.x * per;
    int32_t sum = 0;
    for (int q = 0; q < per; ++q)
        if (q0 + q < m) sum += a[q0 + q];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - sum;
    for (int q = 0; q < per; ++q)
        if (q0 + q < m) {
            const int32_t v = a[q0 + q];
            a[q0 + q] = run;
            run += v;
        }
}

// stable scatter by digit: within a block, rank = earlier keys of the same
// digit (warps in order, lanes in order); vin NULL: the values are the indices
__global__ void __launch_bounds__(RS_BLOCK) rs_scatter_kernel(const uint32_t *kin, const int32_t *vin, uint32_t *kout,
                                                              int32_t *vout, int nt, const int32_t *nt_dev, int shift,
                                                              int nblk, const int32_t *rh)
{
    __shared__ int32_t wc[RS_BLOCK / 32][RS_RADIX];
    const int n = nt_dev ? *nt_dev : nt;
    const int i = blockIdx.x * RS_BLOCK + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < (RS_BLOCK / 32) * RS_RADIX; q += RS_BLOCK) (&wc[0][0])[q] = 0;
    __syncthreads();
    const bool live = i < n;
    const uint32_t k = live ? kin[i] : 0u;
    const int32_t v = live ? (vin ? vin[i] : i) : 0;
    const int dg = (int)((k >> shift) & (RS_RADIX - 1));
    const unsigned peers = __match_any_sync(0xffffffffu, live ? dg : RS_RADIX);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (live && rank == 0) wc[warp][dg] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < RS_RADIX) {
        int32_t run = 0;
        for (int w = 0; w < RS_BLOCK / 32; ++w) {
            const int32_t c = wc[w][threadIdx.x];
            wc[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    if (live) {
        const int dst = rh[dg * nblk + blockIdx.x] + wc[warp][dg] + rank;
        kout[dst] = k;
        vout[dst] = v;
    }
}

// perm = target indices sorted by code, index order within a code; code is
// overwritten; tk / tv scratch of capacity entries, rh of RS_RADIX * nblk + 1
static void binsort(const uint32_t *code_in, uint32_t *code, int32_t *perm, uint32_t *tk, int32_t *tv, int32_t *rh,
                    int nt, const int32_t *nt_dev, int capacity, cudaStream_t s)
{
    const int nblk = obem_binsort_blocks(capacity);
    const uint32_t *kin[3] = {code_in, tk, code};
    const int32_t *vin[3] = {NULL, perm, tv};
    uint32_t *kout[3] = {tk, code, tk};
    int32_t *vout[3] = {perm, tv, perm};
    for (int p = 0; p < 3; ++p) {
        rs_hist_kernel<<<nblk, RS_BLOCK, 0, s>>>(kin[p], nt, nt_dev, 6 * p, nblk, rh);
        rs_scan_kernel<<<1, 1024, 0, s>>>(rh, RS_RADIX * nblk);
        rs_scatter_kernel<<<nblk, RS_BLOCK, 0, s>>>(kin[p], vin[p], kout[p], vout[p], nt, nt_dev, 6 * p, nblk, rh);
    }
}

// Spatial order of n points for a pass that runs over the cells outermost
// (the influence of charges on the cells): the Morton bins of the cell box,
// the stable radix sort and the blocks of at most CT_BLOCK_N points inside a
// super-bin, as for the targets of the cell kernels, in scratch of
// obem_point_bins_bytes(n) bytes.
static size_t pb_align(size_t b) { return (b + 255) & ~(size_t)255; }
int obem_point_bins_maxblocks(int n) { return n / CT_BLOCK_N + 2 + (n < OBEM_NSUPER ? n : OBEM_NSUPER); }
size_t obem_point_bins_bytes(int n)
{
    const size_t e = pb_align(sizeof(int32_t) * (size_t)n);
    return 4 * e + pb_align(sizeof(int32_t) * ((size_t)RS_RADIX * obem_binsort_blocks(n) + 1)) +
           pb_align(sizeof(int32_t) * OBEM_NBINS) + pb_align(sizeof(int2) * obem_point_bins_maxblocks(n)) +
           pb_align(sizeof(int32_t) * 8);
}
int obem_point_bins(obem_ctx *ctx, const float4 *pts, int n, void *scratch, int32_t **perm, int2 **blocks,
                    int32_t **nblocks, cudaStream_t s)
{
    char *p = (char *)scratch;
    const size_t e = pb_align(sizeof(int32_t) * (size_t)n);
    uint32_t *code = (uint32_t *)p; p += e;
    *perm = (int32_t *)p; p += e;
    uint32_t *tk = (uint32_t *)p; p += e;
    int32_t *tv = (int32_t *)p; p += e;
    int32_t *rh = (int32_t *)p; p += pb_align(sizeof(int32_t) * ((size_t)RS_RADIX * obem_binsort_blocks(n) + 1));
    int32_t *hist = (int32_t *)p; p += pb_align(sizeof(int32_t) * OBEM_NBINS);
    *blocks = (int2 *)p; p += pb_align(sizeof(int2) * obem_point_bins_maxblocks(n));
    *nblocks = (int32_t *)p;
    FieldLaunch L;
    memset(&L, 0, sizeof L);
    L.targets = pts;
    L.nt = n;
    float3 lo = make_float3(ctx->bbox_lo[0], ctx->bbox_lo[1], ctx->bbox_lo[2]);
    float3 sc;
    sc.x = (float)OBEM_BINS_PER_AXIS / fmaxf(ctx->bbox_hi[0] - ctx->bbox_lo[0], 1e-30f);
    sc.y = (float)OBEM_BINS_PER_AXIS / fmaxf(ctx->bbox_hi[1] - ctx->bbox_lo[1], 1e-30f);
    sc.z = (float)OBEM_BINS_PER_AXIS / fmaxf(ctx->bbox_hi[2] - ctx->bbox_lo[2], 1e-30f);
    OBEM_CUDA(ctx, cudaMemsetAsync(hist, 0, sizeof(int32_t) * OBEM_NBINS, s));
    bin_count_kernel<<<(n + 255) / 256, 256, 0, s>>>(L, lo, sc, code, hist);
    bin_scan_kernel<<<1, 1024, 0, s>>>(hist);
    block_list_kernel<<<1, 1024, 0, s>>>(hist, n, NULL, *blocks, *nblocks);
    binsort(code, code, *perm, tk, tv, rh, n, NULL, n, s);
    OBEM_LAUNCH(ctx);
    return OBEM_OK;
}

// ---------------------------------------------------------------- cell field kernels
// The cell field is computed by three kernels over the same partition of the
// (binned) targets into blocks of CT_BLOCK targets.  A cell is "near" a block
// if its centroid is closer than 1.5 h to the bounding box of the block's
// targets (or if the block is so spread out that its frame cannot resolve the
// cell); the test is the same function in all three kernels.
//   near_closed_kernel  near cells, targets with d < h: FP64 closed form
//                       (pairs queued per warp, 32 per evaluation); writes
//                       E_out = e_ext + these terms
//   near_quad_kernel    near cells, all other targets: 7-point rule on 16
//                       sub-triangles (<= 2.7e-6 for d >= h), or on 4 (28
//                       points, 2.6e-6 for d >= 1.5 h) for a warp whose whole
//                       box is 1.5 h away; target-centroid differences exact
//   cell_kernel         far cells: 1 / 3 / 4 / 6 / 7 / 28 quadrature points
//                       chosen by the distance to the box, emitted as point
//                       sources in a frame centred on the block and consumed
//                       by the packed f32x2 loop
#define CT_THREADS 128
#define CT_TPT 4
#define CT_BLOCK (CT_THREADS * CT_TPT)
#define CT_CHUNK 32                 // far cells emitted per round
#define CT_MAXPTS (CT_CHUNK * 28 + 4)
#define NEAR_CHUNK 128              // cells tested per round
#define NQ_CELLS 8                  // near cells per quadrature round
#define NQ_PTS 112

#define TIER_28PT_H2 2.25f          // d >= 1.5 h
#define FRAME_H 0.05f               // a cell needs h >= FRAME_H * frame scale to be far



// squared distance from point c to the box [lo, hi]
__device__ __forceinline__ float box_d2(float cx, float cy, float cz, float3 lo, float3 hi)
{
    float dx = fmaxf(fmaxf(lo.x - cx, cx - hi.x), 0.f);
    float dy = fmaxf(fmaxf(lo.y - cy, cy - hi.y), 0.f);
    float dz = fmaxf(fmaxf(lo.z - cz, cz - hi.z), 0.f);
    return dx * dx + dy * dy + dz * dz;
}

struct BlockFrame {
    float3 lo, hi;      // box of the block's targets (absolute)
    float3 o;           // frame origin: box centre if the block is compact, else 0
    float scale2;       // squared largest |target - o| bound (box corners)
};

// This block's range of the (binned) target order: [base, end).  Returns
// false for grid blocks beyond the block list.
__device__ __forceinline__ bool block_range(const FieldLaunch &L, int nt, int &base, int &end)
{
    if (L.blocks) {
        if ((int)blockIdx.x >= *L.nblocks) return false;
        const int2 b = L.blocks[blockIdx.x];
        base = b.x;
        end = b.x + b.y;
    } else {
        base = blockIdx.x * CT_BLOCK;
        end = min(nt, base + CT_BLOCK);
    }
    return base < nt;
}

// This block's cells [poff, poff + np) of the cell arrays: all cells, or in a
// batch of chambers the cells of the block's chamber.
__device__ __forceinline__ void block_cells(const FieldLaunch &L, int &poff, int &np)
{
    poff = 0;
    np = L.panels.np;
    if (L.block_cham) {
        const int2 r = L.cham_pan[L.block_cham[blockIdx.x]];
        poff = r.x;
        np = r.y;
    }
}

// Targets of this block (binned order, absolute coordinates) and its frame.
// Target slot k of thread t is base + k * CT_THREADS + t.
// CONTIG: warp w holds the block's targets w * 32 * CT_TPT ... (consecutive in
// the binned order, so each warp's box is compact) and wlo / whi get it.
template <bool CONTIG = false>
__device__ __forceinline__ void block_targets(const FieldLaunch &L, int end, int base, float *tx, float *ty,
                                              float *tz, int *ti, BlockFrame &F, float3 *wlo = NULL,
                                              float3 *whi = NULL)
{
    __shared__ float red[6][CT_THREADS / 32];
    float mn[3] = {3e38f, 3e38f, 3e38f}, mx[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        int i = CONTIG ? base + (int)(threadIdx.x & ~31u) * CT_TPT + k * 32 + (int)(threadIdx.x & 31u)
                       : base + k * CT_THREADS + threadIdx.x;
        int ic = i < end ? i : (end - 1);
        ti[k] = L.perm ? L.perm[ic] : ic;
        float4 p = L.targets[ti[k]];
        tx[k] = p.x; ty[k] = p.y; tz[k] = p.z;
        if (i >= end) { ti[k] = -1; continue; }
        mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
        mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int q = 16; q; q >>= 1) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], q));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], q));
        }
    if (CONTIG) {
        *wlo = make_float3(mn[0], mn[1], mn[2]);
        *whi = make_float3(mx[0], mx[1], mx[2]);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; ++c) { red[c][w] = mn[c]; red[3 + c][w] = mx[c]; }
    __syncthreads();
    float r[6];
    for (int c = 0; c < 6; ++c) {
        float v = red[c][0];
        for (int q = 1; q < CT_THREADS / 32; ++q) v = c < 3 ? fminf(v, red[c][q]) : fmaxf(v, red[c][q]);
        r[c] = v;
    }
    F.lo = make_float3(r[0], r[1], r[2]);
    F.hi = make_float3(r[3], r[4], r[5]);
    const float hx = 0.5f * (r[3] - r[0]), hy = 0.5f * (r[4] - r[1]), hz = 0.5f * (r[5] - r[2]);
    const float half2 = hx * hx + hy * hy + hz * hz;
    const float ax = fmaxf(fabsf(r[0]), fabsf(r[3])), ay = fmaxf(fabsf(r[1]), fabsf(r[4])),
                az = fmaxf(fabsf(r[2]), fabsf(r[5]));
    const float abs2 = ax * ax + ay * ay + az * az;
    if (half2 <= abs2) {
        F.o = make_float3(0.5f * (r[0] + r[3]), 0.5f * (r[1] + r[4]), 0.5f * (r[2] + r[5]));
        F.scale2 = half2;
    } else {
        F.o = make_float3(0.f, 0.f, 0.f);
        F.scale2 = abs2;
    }
}

// the near test shared by the three cell kernels
__device__ __forceinline__ bool cell_is_near(float4 ca, float h2, const BlockFrame &F)
{
    return box_d2(ca.x, ca.y, ca.z, F.lo, F.hi) < TIER_28PT_H2 * h2 || h2 < (FRAME_H * FRAME_H) * F.scale2;
}

// FP64 closed form of one cell at one target, times k_C sigma (FP32 result)
__device__ __noinline__ float4 closed_val(const double *v, const double *g, float tx, float ty, float tz, float sg)
{
    double phi, Fx, Fy, Fz;
    if (g) tri_closed_form_g(v, g, (double)tx, (double)ty, (double)tz, phi, Fx, Fy, Fz);
    else tri_closed_form(v, (double)tx, (double)ty, (double)tz, phi, Fx, Fy, Fz);
    const double kq = OBEM_KC * (double)sg;
    return make_float4((float)(kq * Fx), (float)(kq * Fy), (float)(kq * Fz), (float)(kq * phi));
}

// deterministic compaction of the near cells of [pb, pb + NEAR_CHUNK) of the
// block's cells into list (as indices of the cell arrays)
__device__ __forceinline__ int near_list(const FieldLaunch &L, int poff, int np, int pb, const BlockFrame &F,
                                         int *list, int *cnt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = pb + threadIdx.x;
    bool near = false;
    if (j < np) near = cell_is_near(L.panels.c_a[poff + j], L.panels.g0_h[poff + j].w, F);
    const unsigned bal = __ballot_sync(0xffffffffu, near);
    __syncthreads();
    if (lane == 0) cnt[warp] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < CT_THREADS / 32; ++w) { if (w < warp) off += cnt[w]; tot += cnt[w]; }
    if (near) list[off + __popc(bal & ((1u << lane) - 1u))] = poff + j;
    __syncthreads();
    return tot;
}

// exact target - centroid difference: (t - c_hi) - c_lo
__device__ __forceinline__ void diff_exact(float t, float chi, float clo, float &d)
{
    d = (t - chi) - clo;
}

// near cells, targets within h of them: FP64 closed form; E_out = e_ext + that.
// Few targets of a warp lie within h of a given cell, and a warp-wide FP64
// instruction costs the same with one lane active as with 32, so the (target,
// cell) pairs are queued per warp and evaluated 32 at a time.  Queue order is
// (cell, target slot, lane) and each lane adds its results in queue order:
// the sums are deterministic.
#define NC_Q 64                     // per-warp queue (< 32 left after a flush, + 32 appended)
__device__ __forceinline__ void nc_flush(const FieldLaunch &L, int n, const float4 *qp, const int *qt, float4 *res,
                                         float (*P)[4])
{
    const int lane = threadIdx.x & 31;
    if (lane < n) {
        const float4 e = qp[lane];
        const int j = __float_as_int(e.w);
        res[lane] = closed_val(L.panels.v64 + 9 * (size_t)j,
                               L.panels.geo ? L.panels.geo + (size_t)OBEM_GEO64 * j : NULL, e.x, e.y, e.z, L.sigma[j]);
    }
    __syncwarp();
    for (int e = 0; e < n; ++e) {
        const int t = qt[e];
        if ((t & 31) != lane) continue;
        const float4 r = res[e];
#pragma unroll
        for (int k = 0; k < CT_TPT; ++k)
            if ((t >> 5) == k) { P[k][0] += r.x; P[k][1] += r.y; P[k][2] += r.z; P[k][3] += r.w; }
    }
    __syncwarp();
}

template <bool WANT_V, bool COUNT>
__global__ void __launch_bounds__(CT_THREADS)
near_closed_kernel(FieldLaunch L)
{
    __shared__ int s_list[NEAR_CHUNK];
    __shared__ int s_cnt[CT_THREADS / 32];
    __shared__ float4 s_qp[CT_THREADS / 32][NC_Q];     // target position, cell index (bits)
    __shared__ int s_qt[CT_THREADS / 32][NC_Q];        // target slot << 5 | owner lane
    __shared__ float4 s_res[CT_THREADS / 32][32];
    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    int base, end;
    if (!block_range(L, nt, base, end)) return;
    float tx[CT_TPT], ty[CT_TPT], tz[CT_TPT];
    int ti[CT_TPT];
    BlockFrame F;
    block_targets(L, end, base, tx, ty, tz, ti, F);
    int poff, np;
    block_cells(L, poff, np);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *qp = s_qp[warp], *res = s_res[warp];
    int *qt = s_qt[warp];
    // warps whose target slots are all padding skip the arithmetic
    const bool warp_live = base + (int)(threadIdx.x & ~31u) < end;
    float S[CT_TPT][4], C[CT_TPT][4], P[CT_TPT][4];
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) { S[k][c] = 0.f; C[k][c] = 0.f; P[k][c] = 0.f; }
    unsigned long long cntA = 0;
    int nq = 0;                                         // queued pairs (warp-uniform)
    for (int pb = 0; pb < np; pb += NEAR_CHUNK) {
        const int tot = near_list(L, poff, np, pb, F, s_list, s_cnt);
        if (tot == 0) continue;
        for (int q = 0; q < (warp_live ? tot : 0); ++q) {
            const int j = s_list[q];
            const float4 ca = L.panels.c_a[j], cl = L.panels.c_lo[j];
            const float h2 = L.panels.g0_h[j].w;
#pragma unroll
            for (int k = 0; k < CT_TPT; ++k) {
                float dx, dy, dz;
                diff_exact(tx[k], ca.x, cl.x, dx); diff_exact(ty[k], ca.y, cl.y, dy); diff_exact(tz[k], ca.z, cl.z, dz);
                const bool hit = ti[k] >= 0 && fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < h2;
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (bal == 0u) continue;
                if (hit) {
                    const int e = nq + __popc(bal & ((1u << lane) - 1u));
                    qp[e] = make_float4(tx[k], ty[k], tz[k], __int_as_float(j));
                    qt[e] = (k << 5) | lane;
                    if (COUNT) ++cntA;
                }
                nq += __popc(bal);
                __syncwarp();
                if (nq >= 32) {
                    nc_flush(L, 32, qp, qt, res, P);
                    nq -= 32;
                    if (lane < nq) { qp[lane] = qp[32 + lane]; qt[lane] = qt[32 + lane]; }
                    __syncwarp();
                }
            }
        }
#pragma unroll
        for (int k = 0; k < CT_TPT; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) { two_sum_acc(S[k][c], C[k][c], P[k][c]); P[k][c] = 0.f; }
    }
    if (nq > 0) {
        nc_flush(L, nq, qp, qt, res, P);
#pragma unroll
        for (int k = 0; k < CT_TPT; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) two_sum_acc(S[k][c], C[k][c], P[k][c]);
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
    if (COUNT && L.counters) atomicAdd(&L.counters[4], cntA);
}

// near cells, targets at d >= h: 112-point rule, exact relative coordinates
template <bool WANT_V, bool COUNT>
__global__ void __launch_bounds__(CT_THREADS)
near_quad_kernel(FieldLaunch L)
{
    __shared__ int s_list[NEAR_CHUNK];
    __shared__ int s_cnt[CT_THREADS / 32];
    __shared__ SrcPk s_off[NQ_CELLS][NQ_PTS];                // offsets from the centroid, weight
    __shared__ SrcPk s_off28[NQ_CELLS][28];                   // the same cells' 28-point rule
    __shared__ float4 s_cell[NQ_CELLS][2];                    // (c_hi, h^2), (c_lo, 0)
    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    int base, end;
    if (!block_range(L, nt, base, end)) return;
    const int tid = threadIdx.x;
    float tx[CT_TPT], ty[CT_TPT], tz[CT_TPT];
    int ti[CT_TPT];
    BlockFrame F;
    float3 wlo, whi;                       // this warp's box: its targets are consecutive
    block_targets<true>(L, end, base, tx, ty, tz, ti, F, &wlo, &whi);
    int poff, np;
    block_cells(L, poff, np);
    const bool warp_live = base + (int)(threadIdx.x & ~31u) * CT_TPT < end;
    float S[CT_TPT][4], C[CT_TPT][4];
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        int ic = ti[k] >= 0 ? ti[k] : 0;
        float4 e = L.E_out[ic];
        S[k][0] = e.x; S[k][1] = e.y; S[k][2] = e.z; S[k][3] = WANT_V ? e.w : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) C[k][c] = 0.f;
    }
    u64 TX[2], TY[2], TZ[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        TX[p] = pk(tx[2 * p], tx[2 * p + 1]);
        TY[p] = pk(ty[2 * p], ty[2 * p + 1]);
        TZ[p] = pk(tz[2 * p], tz[2 * p + 1]);
    }
    unsigned long long cntQ = 0, cntP = 0, cntC = 0;
    int wlive = 0;                                        // live targets of this warp
    if (COUNT)
#pragma unroll
        for (int k = 0; k < CT_TPT; ++k) wlive += __popc(__ballot_sync(0xffffffffu, ti[k] >= 0));
    for (int pb = 0; pb < np; pb += NEAR_CHUNK) {
        const int tot = near_list(L, poff, np, pb, F, s_list, s_cnt);
        for (int g = 0; g < tot; g += NQ_CELLS) {
            const int ng = min(NQ_CELLS, tot - g);
            __syncthreads();
            // quadrature offsets of the group's cells: 112 and 28 points each
            for (int t = tid; t < ng * (NQ_PTS + 28); t += CT_THREADS) {
                const int c = t / (NQ_PTS + 28), kk = t % (NQ_PTS + 28);
                const bool fine = kk < NQ_PTS;
                const int k = fine ? kk : kk - NQ_PTS;
                const int j = s_list[g + c];
                const float4 g0 = L.panels.g0_h[j], g1 = L.panels.g1[j], g2 = L.panels.g2[j];
                float3 off;
                float wf;
                rule_point(fine ? 2 : 1, k, make_float3(g0.x, g0.y, g0.z), make_float3(g1.x, g1.y, g1.z),
                           make_float3(g2.x, g2.y, g2.z), off, wf);
                const float w = L.panels.c_a[j].w * L.sigma[j] * wf;
                SrcPk sp;
                sp.xx = pk(off.x, off.x); sp.yy = pk(off.y, off.y); sp.zz = pk(off.z, off.z); sp.qq = pk(w, w);
                if (fine) s_off[c][k] = sp;
                else s_off28[c][k] = sp;
                if (k == 0) {
                    const float4 ca = L.panels.c_a[j], cl = L.panels.c_lo[j];
                    s_cell[c][0] = make_float4(ca.x, ca.y, ca.z, g0.w);
                    s_cell[c][1] = make_float4(cl.x, cl.y, cl.z, 0.f);
                }
            }
            __syncthreads();
            u64 AX[2], AY[2], AZ[2], AV[2];
#pragma unroll
            for (int p = 0; p < 2; ++p) AX[p] = AY[p] = AZ[p] = AV[p] = 0ull;
            for (int c = 0; c < (warp_live ? ng : 0); ++c) {
                const float4 ch = s_cell[c][0], cl = s_cell[c][1];
                // the 28-point rule (2.6e-6 at 1.5 h) when this warp's whole box is
                // at least 1.5 h from the centroid, else the 112-point rule (warp-uniform)
                const bool coarse = box_d2(ch.x + cl.x, ch.y + cl.y, ch.z + cl.z, wlo, whi) >= TIER_28PT_H2 * ch.w;
                const SrcPk *qp = coarse ? s_off28[c] : s_off[c];
                const int nqp = coarse ? 28 : NQ_PTS;
                if (COUNT && (tid & 31) == 0) { cntP += (unsigned long long)nqp * wlive; cntC += wlive; }
                // exact target - centroid per pack; targets within h get a
                // 1e30 m^2 softening, i.e. no term here (theirs is the closed form)
                u64 DX[2], DY[2], DZ[2], EP[2];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    DX[p] = sub2(sub2(TX[p], pk(ch.x, ch.x)), pk(cl.x, cl.x));
                    DY[p] = sub2(sub2(TY[p], pk(ch.y, ch.y)), pk(cl.y, cl.y));
                    DZ[p] = sub2(sub2(TZ[p], pk(ch.z, ch.z)), pk(cl.z, cl.z));
                    u64 d2 = fma2(DZ[p], DZ[p], fma2(DY[p], DY[p], mul2(DX[p], DX[p])));
                    float da, db;
                    upk(d2, da, db);
                    EP[p] = pk(da < ch.w ? 1e30f : 0.0f, db < ch.w ? 1e30f : 0.0f);
                }
#pragma unroll 4
                for (int k = 0; k < nqp; ++k) {
                    const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(&qp[k].xx);
                    const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&qp[k].zz);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        u64 dx = sub2(DX[p], a.x);
                        u64 dy = sub2(DY[p], a.y);
                        u64 dz = sub2(DZ[p], b.x);
                        u64 r2 = fma2(dx, dx, EP[p]);
                        r2 = fma2(dy, dy, r2);
                        r2 = fma2(dz, dz, r2);
                        float ra, rb;
                        upk(r2, ra, rb);
                        u64 inv = pk(rsq(ra), rsq(rb));
                        u64 s = mul2(b.y, inv);
                        u64 s3 = mul2(s, mul2(inv, inv));
                        AX[p] = fma2(dx, s3, AX[p]);
                        AY[p] = fma2(dy, s3, AY[p]);
                        AZ[p] = fma2(dz, s3, AZ[p]);
                        if (WANT_V) AV[p] = add2(AV[p], s);
                    }
                }
            }
            if (COUNT && tid == 0) cntQ += ng;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float a0, a1;
                upk(AX[p], a0, a1); two_sum_acc(S[2 * p][0], C[2 * p][0], a0); two_sum_acc(S[2 * p + 1][0], C[2 * p + 1][0], a1);
                upk(AY[p], a0, a1); two_sum_acc(S[2 * p][1], C[2 * p][1], a0); two_sum_acc(S[2 * p + 1][1], C[2 * p + 1][1], a1);
                upk(AZ[p], a0, a1); two_sum_acc(S[2 * p][2], C[2 * p][2], a0); two_sum_acc(S[2 * p + 1][2], C[2 * p + 1][2], a1);
                if (WANT_V) { upk(AV[p], a0, a1); two_sum_acc(S[2 * p][3], C[2 * p][3], a0); two_sum_acc(S[2 * p + 1][3], C[2 * p + 1][3], a1); }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        if (ti[k] < 0) continue;
        float4 e;
        e.x = (float)((double)S[k][0] + (double)C[k][0]);
        e.y = (float)((double)S[k][1] + (double)C[k][1]);
        e.z = (float)((double)S[k][2] + (double)C[k][2]);
        e.w = WANT_V ? (float)((double)S[k][3] + (double)C[k][3]) : 0.f;
        L.E_out[ti[k]] = e;
    }
    if (COUNT && L.counters && tid == 0) atomicAdd(&L.counters[3], cntQ);
    if (COUNT && L.counters && (tid & 31) == 0) { atomicAdd(&L.counters[5], cntP); atomicAdd(&L.counters[6], cntC); }
}

// far cells as quadrature-point sources, in the block's frame
template <bool WANT_V, bool COUNT, bool BATCH = false>
__global__ void __launch_bounds__(CT_THREADS)
cell_kernel(FieldLaunch L)
{
    __shared__ SrcPk s_pts[CT_MAXPTS];
    __shared__ PanTile s_pan[CT_CHUNK];
    __shared__ int s_n[CT_CHUNK], s_off[CT_CHUNK + 1];
    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    int base, end;
    if (!block_range(L, nt, base, end)) return;
    float tx[CT_TPT], ty[CT_TPT], tz[CT_TPT];
    int ti[CT_TPT];
    BlockFrame F;
    block_targets(L, end, base, tx, ty, tz, ti, F);
    // warps whose target slots are all padding skip the arithmetic
    const bool warp_live = base + (int)(threadIdx.x & ~31u) < end;
    const float3 o = F.o;
    float S[CT_TPT][4], C[CT_TPT][4];
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        int ic = ti[k] >= 0 ? ti[k] : 0;
        float4 e = L.E_out[ic];                    // near part + e_ext
        S[k][0] = e.x; S[k][1] = e.y; S[k][2] = e.z; S[k][3] = WANT_V ? e.w : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) C[k][c] = 0.f;
    }
    u64 TX[2], TY[2], TZ[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        TX[p] = pk(tx[2 * p] - o.x, tx[2 * p + 1] - o.x);
        TY[p] = pk(ty[2 * p] - o.y, ty[2 * p + 1] - o.y);
        TZ[p] = pk(tz[2 * p] - o.z, tz[2 * p + 1] - o.z);
    }
    unsigned long long cnt1 = 0, cnt3 = 0, cnt7 = 0, cntP = 0, cntC = 0;
    int poff = 0, np = L.panels.np;
    if (BATCH) block_cells(L, poff, np);
    const int tid = threadIdx.x;
    for (int pb = 0; pb < np; pb += CT_CHUNK) {
        __syncthreads();
        if (tid < 32) {
            // warp 0: tier of each cell of the chunk, point counts, offsets
            const int j = poff + pb + tid;
            int n = 0;
            if (pb + tid < np) {
                const float4 ca = L.panels.c_a[j], cl = L.panels.c_lo[j];
                const float sg = L.sigma[j];
                PanTile t;
                t.cq = make_float4((ca.x - o.x) + cl.x, (ca.y - o.y) + cl.y, (ca.z - o.z) + cl.z, ca.w * sg);
                t.g0 = L.panels.g0_h[j];
                t.g1 = L.panels.g1[j];
                t.g2 = L.panels.g2[j];
                s_pan[tid] = t;
                const float h2 = t.g0.w;
                if (!cell_is_near(ca, h2, F)) {
                    const float d2 = box_d2(ca.x, ca.y, ca.z, F.lo, F.hi);
                    n = d2 >= TIER_1PT_H2 * h2 ? 1 : d2 >= TIER_3PT_H2 * h2 ? 3 : d2 >= TIER_4PT_H2 * h2 ? 4
                      : d2 >= TIER_6PT_H2 * h2 ? 6 : d2 >= TIER_7PT_H2 * h2 ? 7 : 28;
                }
            }
            int inc = n;
            for (int q = 1; q < 32; q <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, inc, q);
                if (tid >= q) inc += v;
            }
            s_n[tid] = n;
            s_off[tid] = inc - n;
            if (tid == 31) s_off[CT_CHUNK] = inc;
        }
        __syncthreads();
        const int npts = s_off[CT_CHUNK];
        // emit: 4 threads per cell
        {
            const int c = tid >> 2, sub = tid & 3;
            const int n = s_n[c];
            if (n) {
                const PanTile t = s_pan[c];
                const float q = t.cq.w;
                const float3 G0 = make_float3(t.g0.x, t.g0.y, t.g0.z), G1 = make_float3(t.g1.x, t.g1.y, t.g1.z),
                             G2 = make_float3(t.g2.x, t.g2.y, t.g2.z);
                for (int k = sub; k < n; k += 4) {
                    float3 off;
                    float w;
                    // points c + s g_k (g_k = v_k - c): the symmetric rules' points
                    // (a, b, b) are c + (a - b) g_k since g_0 + g_1 + g_2 = 0
                    float wf;
                    far_point(n, k, G0, G1, G2, off, wf);
                    w = q * wf;
                    const float px = t.cq.x + off.x, py = t.cq.y + off.y, pz = t.cq.z + off.z;
                    SrcPk sp;
                    sp.xx = pk(px, px); sp.yy = pk(py, py); sp.zz = pk(pz, pz); sp.qq = pk(w, w);
                    s_pts[s_off[c] + k] = sp;
                }
            }
            const int pad = (npts + 3) & ~3;
            if (tid < pad - npts) {
                SrcPk sp;
                sp.xx = sp.yy = sp.zz = pk(1e18f, 1e18f);
                sp.qq = pk(0.f, 0.f);
                s_pts[npts + tid] = sp;
            }
        }
        if (COUNT && tid < 32) {
            const int n = s_n[tid];
            cnt1 += n == 1; cnt3 += n >= 3 && n <= 6; cnt7 += n >= 7;
            const unsigned nc = __popc(__ballot_sync(0xffffffffu, n > 0));
            if (tid == 0) { cntP += (unsigned long long)npts * (end - base); cntC += (unsigned long long)nc * (end - base); }
        }
        __syncthreads();
        const int npad = warp_live ? (npts + 3) & ~3 : 0;
        if (npad == 0) continue;
        u64 AX[2], AY[2], AZ[2], AV[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) AX[p] = AY[p] = AZ[p] = AV[p] = 0ull;
#pragma unroll 4
        for (int jj = 0; jj < npad; ++jj) {
            const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(&s_pts[jj].xx);
            const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&s_pts[jj].zz);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                u64 dx = sub2(TX[p], a.x);
                u64 dy = sub2(TY[p], a.y);
                u64 dz = sub2(TZ[p], b.x);
                u64 r2 = mul2(dx, dx);
                r2 = fma2(dy, dy, r2);
                r2 = fma2(dz, dz, r2);
                float ra, rb;
                upk(r2, ra, rb);
                u64 inv = pk(rsq(ra), rsq(rb));
                u64 s = mul2(b.y, inv);
                u64 s3 = mul2(s, mul2(inv, inv));
                AX[p] = fma2(dx, s3, AX[p]);
                AY[p] = fma2(dy, s3, AY[p]);
                AZ[p] = fma2(dz, s3, AZ[p]);
                if (WANT_V) AV[p] = add2(AV[p], s);
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
    }
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        if (ti[k] < 0) continue;
        float4 e;
        e.x = (float)((double)S[k][0] + (double)C[k][0]);
        e.y = (float)((double)S[k][1] + (double)C[k][1]);
        e.z = (float)((double)S[k][2] + (double)C[k][2]);
        e.w = WANT_V ? (float)((double)S[k][3] + (double)C[k][3]) : 0.f;
        L.E_out[ti[k]] = e;
    }
    if (COUNT && L.counters) {
        atomicAdd(&L.counters[1], cnt1);
        atomicAdd(&L.counters[2], cnt3);
        atomicAdd(&L.counters[3], cnt7);
        if (tid == 0) { atomicAdd(&L.counters[5], cntP); atomicAdd(&L.counters[6], cntC); }
    }
}

// ---------------------------------------------------------------- far cells in groups
// cell_kernel with the cells visited group by group (CellGroups): a group
// whose centre is at least sqrt(OBEM_GRP_THETA2) radii from the block's box,
// and none of whose cells is too small for the block's frame, is emitted as
// its OBEM_GRP_M equivalent charges; any other group's cells take the
// per-cell tiers of cell_kernel.  A separated group holds no near cell: its
// cells' centroids are >= 8 R from the box and no edge is longer than 2 R,
// so each is > 4 h away, and its smallest h^2 passes the frame test; the
// near kernels and this one therefore split the cells as with cell_kernel.
// Points are gathered in s_pts and consumed by the packed loop when the
// buffer is full, in group order (deterministic).
template <bool WANT_V, bool COUNT>
__global__ void __launch_bounds__(CT_THREADS)
cell_group_kernel(FieldLaunch L, CellGroups G)
{
    __shared__ SrcPk s_pts[CT_MAXPTS];
    __shared__ PanTile s_pan[CT_CHUNK];
    __shared__ int s_n[CT_CHUNK], s_off[CT_CHUNK + 1];
    static_assert(OBEM_GRP_K == CT_CHUNK, "a non-separated group is one per-cell round");
    static_assert(OBEM_GRP_M <= CT_THREADS, "one thread per equivalent charge");
    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    int base, end;
    if (!block_range(L, nt, base, end)) return;
    float tx[CT_TPT], ty[CT_TPT], tz[CT_TPT];
    int ti[CT_TPT];
    BlockFrame F;
    block_targets(L, end, base, tx, ty, tz, ti, F);
    const bool warp_live = base + (int)(threadIdx.x & ~31u) < end;
    const float3 o = F.o;
    float S[CT_TPT][4], C[CT_TPT][4];
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        int ic = ti[k] >= 0 ? ti[k] : 0;
        float4 e = L.E_out[ic];                    // near part + e_ext
        S[k][0] = e.x; S[k][1] = e.y; S[k][2] = e.z; S[k][3] = WANT_V ? e.w : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) C[k][c] = 0.f;
    }
    u64 TX[2], TY[2], TZ[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        TX[p] = pk(tx[2 * p] - o.x, tx[2 * p + 1] - o.x);
        TY[p] = pk(ty[2 * p] - o.y, ty[2 * p + 1] - o.y);
        TZ[p] = pk(tz[2 * p] - o.z, tz[2 * p + 1] - o.z);
    }
    unsigned long long cnt1 = 0, cnt3 = 0, cnt7 = 0, cntP = 0, cntC = 0;
    const int np = L.panels.np;
    const int tid = threadIdx.x;
    int npend = 0;                                 // points waiting in s_pts[0, npend)
    // the packed loop over s_pts[0, n) (padded to a multiple of 4); every
    // thread calls it, and it leaves s_pts free for reuse
    auto consume = [&](int n) {
        if (COUNT && tid == 0) cntP += (unsigned long long)n * (end - base);
        const int npad = (n + 3) & ~3;
        if (tid < npad - n) {
            SrcPk sp;
            sp.xx = sp.yy = sp.zz = pk(1e18f, 1e18f);
            sp.qq = pk(0.f, 0.f);
            s_pts[n + tid] = sp;
        }
        __syncthreads();
        if (warp_live && npad > 0) {
            u64 AX[2], AY[2], AZ[2], AV[2];
#pragma unroll
            for (int p = 0; p < 2; ++p) AX[p] = AY[p] = AZ[p] = AV[p] = 0ull;
#pragma unroll 4
            for (int jj = 0; jj < npad; ++jj) {
                const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(&s_pts[jj].xx);
                const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&s_pts[jj].zz);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    u64 dx = sub2(TX[p], a.x);
                    u64 dy = sub2(TY[p], a.y);
                    u64 dz = sub2(TZ[p], b.x);
                    u64 r2 = mul2(dx, dx);
                    r2 = fma2(dy, dy, r2);
                    r2 = fma2(dz, dz, r2);
                    float ra, rb;
                    upk(r2, ra, rb);
                    u64 inv = pk(rsq(ra), rsq(rb));
                    u64 sq = mul2(b.y, inv);
                    u64 s3 = mul2(sq, mul2(inv, inv));
                    AX[p] = fma2(dx, s3, AX[p]);
                    AY[p] = fma2(dy, s3, AY[p]);
                    AZ[p] = fma2(dz, s3, AZ[p]);
                    if (WANT_V) AV[p] = add2(AV[p], sq);
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
        }
        __syncthreads();
    };
    for (int g = 0; g < G.ng; ++g) {
        const float4 cr = G.cr[g];
        const float gd2 = box_d2(cr.x, cr.y, cr.z, F.lo, F.hi);
        const bool sep = gd2 >= OBEM_GRP_THETA2 * (cr.w * cr.w) && G.h2min[g] >= (FRAME_H * FRAME_H) * F.scale2;
        if (sep) {
            // the group as its equivalent charges at c + R u_k
            if (npend + OBEM_GRP_M > CT_MAXPTS - 4) { consume(npend); npend = 0; }
            if (tid < OBEM_GRP_M) {
                const float4 u = G.u[tid];
                const float w = G.q[(size_t)g * OBEM_GRP_M + tid];
                const float px = (cr.x - o.x) + cr.w * u.x, py = (cr.y - o.y) + cr.w * u.y,
                            pz = (cr.z - o.z) + cr.w * u.z;
                SrcPk sp;
                sp.xx = pk(px, px); sp.yy = pk(py, py); sp.zz = pk(pz, pz); sp.qq = pk(w, w);
                s_pts[npend + tid] = sp;
            }
            npend += OBEM_GRP_M;
            if (COUNT && tid == 0) cntC += (unsigned long long)OBEM_GRP_K * (end - base);
            continue;
        }
        // the group's cells with the per-cell tiers (as one round of cell_kernel)
        __syncthreads();
        if (tid < 32) {
            const int slot = g * OBEM_GRP_K + tid;
            int n = 0;
            if (slot < np) {
                const int j = G.perm[slot];
                const float4 ca = L.panels.c_a[j], cl = L.panels.c_lo[j];
                const float sg = L.sigma[j];
                PanTile t;
                t.cq = make_float4((ca.x - o.x) + cl.x, (ca.y - o.y) + cl.y, (ca.z - o.z) + cl.z, ca.w * sg);
                t.g0 = L.panels.g0_h[j];
                t.g1 = L.panels.g1[j];
                t.g2 = L.panels.g2[j];
                s_pan[tid] = t;
                const float h2 = t.g0.w;
                if (!cell_is_near(ca, h2, F)) {
                    const float d2 = box_d2(ca.x, ca.y, ca.z, F.lo, F.hi);
                    n = d2 >= TIER_1PT_H2 * h2 ? 1 : d2 >= TIER_3PT_H2 * h2 ? 3 : d2 >= TIER_4PT_H2 * h2 ? 4
                      : d2 >= TIER_6PT_H2 * h2 ? 6 : d2 >= TIER_7PT_H2 * h2 ? 7 : 28;
                }
            }
            int inc = n;
            for (int q = 1; q < 32; q <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, inc, q);
                if (tid >= q) inc += v;
            }
            s_n[tid] = n;
            s_off[tid] = inc - n;
            if (tid == 31) s_off[CT_CHUNK] = inc;
        }
        __syncthreads();
        const int npts = s_off[CT_CHUNK];
        if (npend + npts > CT_MAXPTS - 4) { consume(npend); npend = 0; }
        {
            const int c = tid >> 2, sub = tid & 3;
            const int n = s_n[c];
            if (n) {
                const PanTile t = s_pan[c];
                const float q = t.cq.w;
                const float3 G0 = make_float3(t.g0.x, t.g0.y, t.g0.z), G1 = make_float3(t.g1.x, t.g1.y, t.g1.z),
                             G2 = make_float3(t.g2.x, t.g2.y, t.g2.z);
                for (int k = sub; k < n; k += 4) {
                    float3 off;
                    float w;
                    float wf;
                    far_point(n, k, G0, G1, G2, off, wf);
                    w = q * wf;
                    const float px = t.cq.x + off.x, py = t.cq.y + off.y, pz = t.cq.z + off.z;
                    SrcPk sp;
                    sp.xx = pk(px, px); sp.yy = pk(py, py); sp.zz = pk(pz, pz); sp.qq = pk(w, w);
                    s_pts[npend + s_off[c] + k] = sp;
                }
            }
        }
        if (COUNT && tid < 32) {
            const int n = s_n[tid];
            cnt1 += n == 1; cnt3 += n >= 3 && n <= 6; cnt7 += n >= 7;
            const unsigned nc = __popc(__ballot_sync(0xffffffffu, n > 0));
            if (tid == 0) cntC += (unsigned long long)nc * (end - base);
        }
        npend += npts;
    }
    consume(npend);
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        if (ti[k] < 0) continue;
        float4 e;
        e.x = (float)((double)S[k][0] + (double)C[k][0]);
        e.y = (float)((double)S[k][1] + (double)C[k][1]);
        e.z = (float)((double)S[k][2] + (double)C[k][2]);
        e.w = WANT_V ? (float)((double)S[k][3] + (double)C[k][3]) : 0.f;
        L.E_out[ti[k]] = e;
    }
    if (COUNT && L.counters) {
        atomicAdd(&L.counters[1], cnt1);
        atomicAdd(&L.counters[2], cnt3);
        atomicAdd(&L.counters[3], cnt7);
        if (tid == 0) { atomicAdd(&L.counters[5], cntP); atomicAdd(&L.counters[6], cntC); }
    }
}

// ---------------------------------------------------------------- all-pairs kernel
// E_out[i] = init + k_C sum_{p != i} q_p (r_i - r_p) / (|r_i - r_p|^2 + eps^2)^(3/2)
// init = E_out[i] when the cell kernels ran first (ADD), else e_ext.
// One CTA per block of FT_BLOCK_TARGETS targets; each thread holds FT_TPT
// targets as FT_NP packs of two.  The compensated accumulators and the
// recombination proposals live in shared memory (touched once per tile /
// rarely), which keeps the register count low enough for FT_MINB resident
// blocks per SM.
#define FT_NP (FT_TPT / 2)

template <bool WANT_V, bool ADD>
__global__ void __launch_bounds__(FT_THREADS, FT_MINB)
nbody_kernel(FieldLaunch L)
{
    __shared__ SrcPk s_src[FT_SRC_TILE];
    __shared__ float s_acc[2][WANT_V ? 4 : 3][FT_TPT][FT_THREADS];   // [S|C][component][target][thread]

    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    const int ns = L.ns_dev ? *L.ns_dev : L.ns;
    const int base = blockIdx.x * FT_BLOCK_TARGETS;
    if (base >= nt) return;
    const int tid = threadIdx.x;
    constexpr int NC = WANT_V ? 4 : 3;

    u64 TX[FT_NP], TY[FT_NP], TZ[FT_NP];
#pragma unroll
    for (int k = 0; k < FT_TPT; ++k) {
        int i = base + k * FT_THREADS + tid;
        int ic = i < nt ? i : (nt - 1);
        float4 p = L.targets[ic];
        if (k & 1) {
            TX[k >> 1] = pk(__uint_as_float((uint32_t)TX[k >> 1]), p.x);
            TY[k >> 1] = pk(__uint_as_float((uint32_t)TY[k >> 1]), p.y);
            TZ[k >> 1] = pk(__uint_as_float((uint32_t)TZ[k >> 1]), p.z);
        } else {
            TX[k >> 1] = (u64)__float_as_uint(p.x);
            TY[k >> 1] = (u64)__float_as_uint(p.y);
            TZ[k >> 1] = (u64)__float_as_uint(p.z);
        }
        float e[4];
        if (ADD) {
            float4 q = L.E_out[ic];
            e[0] = q.x; e[1] = q.y; e[2] = q.z; e[3] = q.w;
        } else {
            e[0] = L.e_ext.x; e[1] = L.e_ext.y; e[2] = L.e_ext.z; e[3] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) { s_acc[0][c][k][tid] = e[c]; s_acc[1][c][k][tid] = 0.f; }
    }

    const float kC = (float)OBEM_KC;
    const u64 EPS2 = pk(L.eps2, L.eps2);
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
        const bool diag = L.self_exclude && sb < base + L.self_off + FT_BLOCK_TARGETS &&
                          base + L.self_off < sb + FT_SRC_TILE;
        float part[FT_TPT][4];
        if (!diag) {
            u64 AX[FT_NP], AY[FT_NP], AZ[FT_NP], AV[FT_NP];
#pragma unroll
            for (int p = 0; p < FT_NP; ++p) AX[p] = AY[p] = AZ[p] = AV[p] = 0ull;
            FT_UNROLL_BY(FT_UNROLL)
            for (int jj = 0; jj < FT_SRC_TILE; ++jj) {
                const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(&s_src[jj].xx);
                const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&s_src[jj].zz);
#pragma unroll
                for (int p = 0; p < FT_NP; ++p) {
                    u64 dx = sub2(TX[p], a.x);
                    u64 dy = sub2(TY[p], a.y);
                    u64 dz = sub2(TZ[p], b.x);
                    u64 r2 = fma2(dx, dx, EPS2);
                    r2 = fma2(dy, dy, r2);
                    r2 = fma2(dz, dz, r2);
                    float ra, rb;
                    upk(r2, ra, rb);
                    u64 inv = pk(rsq(ra), rsq(rb));
                    u64 s = mul2(b.y, inv);
                    u64 s3 = mul2(s, mul2(inv, inv));
                    AX[p] = fma2(dx, s3, AX[p]);
                    AY[p] = fma2(dy, s3, AY[p]);
                    AZ[p] = fma2(dz, s3, AZ[p]);
                    if (WANT_V) AV[p] = add2(AV[p], s);
                }
            }
#pragma unroll
            for (int p = 0; p < FT_NP; ++p) {
                upk(AX[p], part[2 * p][0], part[2 * p + 1][0]);
                upk(AY[p], part[2 * p][1], part[2 * p + 1][1]);
                upk(AZ[p], part[2 * p][2], part[2 * p + 1][2]);
                if (WANT_V) upk(AV[p], part[2 * p][3], part[2 * p + 1][3]);
            }
        } else {
            // tile holding some of this block's own targets: skip the self pair
#pragma unroll
            for (int k = 0; k < FT_TPT; ++k) { part[k][0] = part[k][1] = part[k][2] = part[k][3] = 0.f; }
            for (int jj = 0; jj < FT_SRC_TILE; ++jj) {
                const int j = sb + jj;
                float sx, sy, sz, sq, dum;
                upk(s_src[jj].xx, sx, dum); upk(s_src[jj].yy, sy, dum);
                upk(s_src[jj].zz, sz, dum); upk(s_src[jj].qq, sq, dum);
#pragma unroll
                for (int k = 0; k < FT_TPT; ++k) {
                    if (j == base + L.self_off + k * FT_THREADS + tid) continue;
                    float txk, tyk, tzk, t2;
                    if (k & 1) { upk(TX[k >> 1], t2, txk); upk(TY[k >> 1], t2, tyk); upk(TZ[k >> 1], t2, tzk); }
                    else { upk(TX[k >> 1], txk, t2); upk(TY[k >> 1], tyk, t2); upk(TZ[k >> 1], tzk, t2); }
                    float dx = __fsub_rn(txk, sx), dy = __fsub_rn(tyk, sy), dz = __fsub_rn(tzk, sz);
                    float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, L.eps2)));
                    float inv = rsq(r2);
                    float s = sq * inv;
                    float s3 = s * (inv * inv);
                    part[k][0] = fmaf(dx, s3, part[k][0]);
                    part[k][1] = fmaf(dy, s3, part[k][1]);
                    part[k][2] = fmaf(dz, s3, part[k][2]);
                    part[k][3] += s;
                }
            }
        }
        // fold the tile's partial sums into the compensated accumulators
#pragma unroll
        for (int k = 0; k < FT_TPT; ++k)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float sv = s_acc[0][c][k][tid], cv = s_acc[1][c][k][tid];
                two_sum_acc(sv, cv, part[k][c]);
                s_acc[0][c][k][tid] = sv;
                s_acc[1][c][k][tid] = cv;
            }
    }

#pragma unroll
    for (int k = 0; k < FT_TPT; ++k) {
        int i = base + k * FT_THREADS + tid;
        if (i >= nt) continue;
        float4 e;
        e.x = (float)((double)s_acc[0][0][k][tid] + (double)s_acc[1][0][k][tid]);
        e.y = (float)((double)s_acc[0][1][k][tid] + (double)s_acc[1][1][k][tid]);
        e.z = (float)((double)s_acc[0][2][k][tid] + (double)s_acc[1][2][k][tid]);
        e.w = WANT_V ? (float)((double)s_acc[0][NC - 1][k][tid] + (double)s_acc[1][NC - 1][k][tid]) : 0.f;
        L.E_out[i] = e;
    }
}

// ---------------------------------------------------------------- symmetric all-pairs kernel
// When the targets are the sources (self_exclude), every unordered pair is
// evaluated once and its reaction is applied to the other charge (Newton's
// third law): per ordered pair 8 FP32 lane-operations and half an rsqrt
// instead of 12 and one.  (The recombination partner search runs separately,
// by spatial hashing, in the step.)
//
// Charges are cut into tiles of SY_T = 1024.  Item (I, d) pairs tile I with
// tile J = (I + d) mod n for d = 0 .. h_I (d = 0: the tile with itself, done
// as ordered pairs); with h_I = floor(n/2), minus one for I >= n/2 when n is
// even, every unordered tile pair occurs exactly once.  A work unit is SY_CH
// consecutive items of one row; persistent blocks take units from a counter.
// Inside an off-diagonal item each warp holds 256 targets (8 per lane, four
// f32x2 packs) and walks the sources of tile J in rounds of 32: the 32
// sources sit one per lane and rotate around the warp by shuffles, carrying
// their own reaction sums, so no reduction is needed; the four warps take
// different 32-source groups in every round and add their sums into shared
// memory in a fixed order.  Every unit writes its target-side sums (Ipart) and
// every item its source-side sums (Jpart) to slots of its own, and
// nbsym_fold_kernel adds them per charge in a fixed order: the result does
// not depend on which block ran which unit.
#ifndef SY_THREADS
#define SY_THREADS 128
#endif
#ifndef SY_MINB
#define SY_MINB 3              // resident blocks per SM the register budget is cut for
#endif
#define SY_NI 8
#define SY_NP (SY_NI / 2)
#define SY_T (SY_THREADS * SY_NI)
#define SY_WARPS (SY_THREADS / 32)
#define SY_NG (SY_T / 32)      // 32-source groups of a tile (rounds of an item)
#define SY_CH 16
#define SY_CH_SMALL 1
#define SY_SMALL_TILES 32      // sets of at most 32 tiles (32768 charges) use single-item units
#define SY_CH_MID 4
#define SY_MID_TILES 256       // and of at most 256 tiles units of 4 items
#define SY_FOLD 8              // rounds (of 32 sources) between compensated folds
#define SY_DTILE 256           // staged sources of the d = 0 item
// The kernel works on positions scaled by 2^40 and charges (k_C q) by 2^80:
// inv = 1/r then carries 2^-40 and inv^3 2^-120, which keeps every product
// finite down to r ~ 1e-20 m (unscaled, inv^3 overflows below 1.4e-13 m); each
// k_C q inv^3 d comes out unscaled, the potential k_C q inv carries 2^40.
// Power-of-two scaling is exact: the results are those of the unscaled sums.
#define SY_XS 1099511627776.0f               // 2^40
#define SY_QS 1208925819614629174706176.0f   // 2^80
#define SY_VS 9.094947017729282e-13f         // 2^-40

struct SymGeom {
    int n, hmax, nch;
};
// CH: items per work unit (SY_CH; SY_CH_SMALL for a set of at most
// SY_SMALL_TILES tiles, so that its few tile pairs still spread over the SMs)
template <int CH>
__host__ __device__ inline SymGeom sym_geom_ch(int nt)
{
    SymGeom g;
    g.n = (nt + SY_T - 1) / SY_T;
    g.hmax = g.n / 2;
    g.nch = (g.hmax + 1 + CH - 1) / CH;
    return g;
}
__host__ __device__ inline SymGeom sym_geom(int nt) { return sym_geom_ch<SY_CH>(nt); }
// off-diagonal items of row I
__host__ __device__ inline int sym_h(const SymGeom &g, int I)
{
    if (g.n & 1) return g.hmax;
    return I < g.n / 2 ? g.hmax : g.hmax - 1;
}

// Partial-sum slots of a launch, one whole set of charges or one pass over a
// range of diagonals: units (I, kch) for kch in [kch_lo, kch_lo + kch_n), the
// target-side sums of unit (I, kch) in slot I * kch_n + (kch - kch_lo), the
// source-side sums of item (I, d) in slot I * jd + (d - kch_lo * SY_CH).
// kch_n == 0: every unit of each chamber (batch of chambers), jd = hmax + 1.
// first / last: the fold starts from the initial field / writes the result;
// otherwise it reads / writes the per-charge FP64 accumulator acc.
struct SymPass {
    int kch_lo, kch_n, jd, first, last;
    double *acc;           // [capacity][4]
};
#define SY_PASS_CH 32      // units (of SY_CH diagonals) per pass: 512 diagonals

size_t obem_sym_jpart_floats(int capacity)
{
    const SymGeom g = sym_geom(capacity);
    return (size_t)g.n * (g.hmax + 1) * 4 * SY_T;
}
size_t obem_sym_ipart_floats(int capacity)
{
    const SymGeom g = sym_geom(capacity);
    return (size_t)g.n * g.nch * 8 * SY_T;
}
// the same for one pass of SY_PASS_CH units per row (the single-context path)
size_t obem_sym_pass_jpart_floats(int capacity)
{
    const SymGeom g = sym_geom(capacity);
    const int jd = g.hmax + 1 < SY_PASS_CH * SY_CH ? g.hmax + 1 : SY_PASS_CH * SY_CH;
    return (size_t)g.n * jd * 4 * SY_T;
}
size_t obem_sym_pass_ipart_floats(int capacity)
{
    const SymGeom g = sym_geom(capacity);
    size_t f = (size_t)g.n * (g.nch < SY_PASS_CH ? g.nch : SY_PASS_CH) * 8 * SY_T;
    if (g.n <= SY_MID_TILES) {
        const SymGeom g1 = g.n <= SY_SMALL_TILES ? sym_geom_ch<SY_CH_SMALL>(capacity) : sym_geom_ch<SY_CH_MID>(capacity);
        const size_t f1 = (size_t)g1.n * (g1.nch < SY_PASS_CH ? g1.nch : SY_PASS_CH) * 8 * SY_T;
        f = f1 > f ? f1 : f;
    }
    return f;
}

// dynamic shared memory of nbsym_kernel: target-side S and C [NC][SY_NI][SY_THREADS]
// each, source-side S and C [NC][SY_T] each (reused as the d = 0 staging tile)
__host__ __device__ constexpr size_t sym_smem(int nc)
{
    return (size_t)2 * nc * SY_NI * SY_THREADS * 4 + (size_t)2 * nc * SY_T * 4;
}

// The kernel runs on a copy of the charges ordered by charge value: negative
// charges first, each class in index order (a stable partition).  Then every
// tile but the one holding the boundary (and the padded last tile) has one
// charge value, and for a pair of such tiles the charges factor out of the
// sums: the inner loop accumulates inv^3 d and the tile's k_C q multiplies the
// sums once (two multiplications fewer per pair).
#define SP_BLOCK 1024
int obem_sym_part_blocks(int capacity) { return (capacity + SP_BLOCK - 1) / SP_BLOCK; }
int obem_sym_tiles(int capacity) { return sym_geom(capacity).n; }

// Partition and tiles of one set of charges (SymBatch.nb == 0: the launch's
// targets, nt or *nt_dev of them) or of a batch of chambers (chamber c holds
// slots [seg_off[c], seg_off[c + 1]), n[c] live, offsets multiples of SY_T):
// slot block b (SP_BLOCK == SY_T slots) belongs to chamber c, whose live
// charges are slots [off, off + n).
__device__ __forceinline__ void sym_block_range(const SymBatch &SB, int nt, const int32_t *nt_dev, int b, int &c,
                                                int &off, int &n)
{
    if (SB.nb) {
        c = SB.slot_cham[b];
        off = SB.seg_off[c];
        n = SB.n[c];
    } else {
        c = 0;
        off = 0;
        n = nt_dev ? *nt_dev : nt;
    }
}

// negative charges per block of SP_BLOCK slots
__global__ void sym_part_count_kernel(const float4 *src, int nt, const int32_t *nt_dev, SymBatch SB, int32_t *bcnt)
{
    int c, off, n;
    sym_block_range(SB, nt, nt_dev, blockIdx.x, c, off, n);
    const int i = blockIdx.x * SP_BLOCK + threadIdx.x;
    const int cnt = __syncthreads_count(i - off < n && src[i].w < 0.f);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = cnt;
}

// exclusive scan of the block counts of one chamber (one block of 1024 per
// chamber; the blocks [0, nb) when there is no batch), in place; the
// chamber's total to tot[c]
__global__ void sym_part_scan_kernel(int32_t *bcnt, int nb, SymBatch SB, int32_t *tot)
{
    __shared__ int32_t part[1024];
    int b0 = 0, b1 = nb;
    if (SB.nb) {
        b0 = SB.seg_off[blockIdx.x] / SP_BLOCK;
        b1 = SB.seg_off[blockIdx.x + 1] / SP_BLOCK;
    }
    const int m = b1 - b0;
    const int per = (m + 1023) / 1024, q0 = b0 + threadIdx.x * per;
    int32_t s = 0;
    for (int q = 0; q < per; ++q)
        if (q0 + q < b1) s += bcnt[q0 + q];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int q = 0; q < per; ++q)
        if (q0 + q < b1) {
            const int32_t v = bcnt[q0 + q];
            bcnt[q0 + q] = run;
            run += v;
        }
    if (threadIdx.x == 1023) tot[blockIdx.x] = part[1023];
}

// sorted[dst] = (position of target i, charge of source i), perm[dst] = i
// (slots of the concatenated arrays; each chamber sorted within its segment)
__global__ void sym_part_scatter_kernel(const float4 *tgt, const float4 *src, int nt, const int32_t *nt_dev,
                                        SymBatch SB, const int32_t *bcnt, const int32_t *tot, float4 *sorted,
                                        int32_t *perm)
{
    __shared__ int32_t wneg[SP_BLOCK / 32];
    int c, off, n;
    sym_block_range(SB, nt, nt_dev, blockIdx.x, c, off, n);
    const int i = blockIdx.x * SP_BLOCK + threadIdx.x;      // slot
    const int li = i - off;                                  // index in the chamber
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    float q = 0.f;
    if (li < n) { p = tgt[i]; q = src[i].w; }
    const bool neg = li < n && q < 0.f;
    const unsigned bal = __ballot_sync(0xffffffffu, neg);
    if (lane == 0) wneg[warp] = __popc(bal);
    __syncthreads();
    int rneg = __popc(bal & ((1u << lane) - 1u));        // negative charges before i in the block
    for (int w = 0; w < warp; ++w) rneg += wneg[w];
    if (li < n) {
        const int negoff = bcnt[blockIdx.x];
        const int lb = blockIdx.x * SP_BLOCK - off;          // the block's first index in the chamber
        const int dst = neg ? negoff + rneg : tot[c] + (lb - negoff) + ((int)threadIdx.x - rneg);
        sorted[off + dst] = make_float4(p.x * SY_XS, p.y * SY_XS, p.z * SY_XS, q);   // positions x 2^40
        perm[off + dst] = i;
    }
}

// per tile of SY_T sorted slots: the common charge, or NaN; slots past n count as 0
__global__ void sym_tileq_kernel(const float4 *sorted, int nt, const int32_t *nt_dev, SymBatch SB, float *tileq)
{
    int c, off, n;
    sym_block_range(SB, nt, nt_dev, blockIdx.x, c, off, n);
    const int base = blockIdx.x * SY_T;
    if (base - off >= n) return;
    const float q0 = sorted[base].w;
    bool same = true;
    for (int k = threadIdx.x; k < SY_T; k += blockDim.x) {
        const int i = base + k;
        same = same && ((i - off < n ? sorted[i].w : 0.f) == q0);
    }
    same = __syncthreads_and(same);
    if (threadIdx.x == 0) tileq[blockIdx.x] = same ? q0 : __int_as_float(0x7fc00000);
}

// units of every chamber of a batch and their offsets (one block)
__global__ void sym_units_kernel(SymBatch SB)
{
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < SB.nb; c0 += 1024) {
        const int c = c0 + threadIdx.x;
        int32_t u = 0;
        if (c < SB.nb && SB.n[c] > 0) {
            const SymGeom G = sym_geom(SB.n[c]);
            u = G.n * G.nch;
        }
        // inclusive block scan
        __shared__ int32_t part[1024];
        part[threadIdx.x] = u;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        if (c < SB.nb) SB.uoff[c] = carry + part[threadIdx.x] - u;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) SB.uoff[SB.nb] = carry;
}

template <bool B> struct SyBool { static constexpr bool value = B; };

template <bool WANT_V, bool BATCH, int CH = SY_CH>
__global__ void __launch_bounds__(SY_THREADS, SY_MINB)
nbsym_kernel(FieldLaunch L, float *jpart, float *ipart, int *counter, const float *tileq, SymBatch SB, SymPass PS)
{
    constexpr int NC = WANT_V ? 4 : 3;
    extern __shared__ __align__(16) unsigned char sy_smem[];
    typedef float TS[SY_NI][SY_THREADS];
    TS *s_S = reinterpret_cast<TS *>(sy_smem);                                   // [NC]
    TS *s_C = s_S + NC;                                                           // [NC]
    float *s_jS = reinterpret_cast<float *>(s_C + NC);                            // [NC * SY_T]
    float *s_jC = s_jS + NC * SY_T;
    SrcPk *s_src = reinterpret_cast<SrcPk *>(s_jS);
    __shared__ int s_unit, s_off, s_nt;
    __shared__ long long s_joff, s_ioff;

    // one set of charges: nt of them, units fixed; a batch: per unit, its
    // chamber's slots [s_off, s_off + s_nt) and partial-sum offsets
    int units, nt0 = 0;
    SymGeom G0;
    if (BATCH) {
        units = SB.uoff[SB.nb];
    } else {
        nt0 = L.nt_dev ? *L.nt_dev : L.nt;
        if (nt0 <= 0) return;
        G0 = sym_geom_ch<CH>(nt0);
        units = G0.n * max(0, min(PS.kch_n, G0.nch - PS.kch_lo));
    }
    // this launch's units of a row and its slot strides (one set of charges)
    const int kn0 = BATCH ? 1 : max(1, min(PS.kch_n, G0.nch - PS.kch_lo)), klo0 = BATCH ? 0 : PS.kch_lo,
              jd0 = BATCH ? 1 : PS.jd;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // k_C x 2^80 (kCs q is k_C q scaled exactly); L.eps2 comes in the scaled
    // positions' units (x 2^80) from the launch
    const float kCs = (float)OBEM_KC * SY_QS;
    const u64 EPS2 = pk(L.eps2, L.eps2);

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const int u = atomicAdd(counter, 1);
            if (BATCH) {
                int lu = -1;
                if (u < units) {
                    int lo = 0, hi = SB.nb;              // uoff[lo] <= u < uoff[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (SB.uoff[mid] <= u) lo = mid; else hi = mid;
                    }
                    lu = u - SB.uoff[lo];
                    s_off = SB.seg_off[lo];
                    s_nt = SB.n[lo];
                    s_joff = SB.joff[lo];
                    s_ioff = SB.ioff[lo];
                }
                s_unit = lu;
            } else {
                s_unit = u < units ? u : -1;
            }
        }
        __syncthreads();
        const int unit = s_unit;
        if (unit < 0) break;
        const int off = BATCH ? s_off : 0;
        const int lim = BATCH ? off + s_nt : nt0;        // end of the live slots
        const SymGeom G = BATCH ? sym_geom_ch<CH>(s_nt) : G0;
        // this launch's units of row I: all (batch) or the pass's range
        const int kn = BATCH ? G.nch : kn0;
        const int klo = BATCH ? 0 : klo0;
        const int jd = BATCH ? G.hmax + 1 : jd0;
        const int I = unit / kn, kch = klo + unit % kn;
        const int d0 = kch * CH, d1 = min(d0 + CH, sym_h(G, I) + 1);
        const int base = off + I * SY_T;
        // targets of tile I: 8 per thread (k * 128 + tid), four packs
        u64 TX[SY_NP], TY[SY_NP], TZ[SY_NP], QI[SY_NP];
#pragma unroll
        for (int k = 0; k < SY_NI; ++k) {
            const int i = base + k * SY_THREADS + tid;
            // position from the targets, charge from the sources (the same charges)
            const float4 p = i < lim ? L.targets[i] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
            const float kq = i < lim ? kCs * L.sources[i].w : 0.f;
            if (k & 1) {
                TX[k >> 1] = pk(__uint_as_float((uint32_t)TX[k >> 1]), p.x);
                TY[k >> 1] = pk(__uint_as_float((uint32_t)TY[k >> 1]), p.y);
                TZ[k >> 1] = pk(__uint_as_float((uint32_t)TZ[k >> 1]), p.z);
                QI[k >> 1] = pk(__uint_as_float((uint32_t)QI[k >> 1]), kq);
            } else {
                TX[k >> 1] = (u64)__float_as_uint(p.x);
                TY[k >> 1] = (u64)__float_as_uint(p.y);
                TZ[k >> 1] = (u64)__float_as_uint(p.z);
                QI[k >> 1] = (u64)__float_as_uint(kq);
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) { s_S[c][k][tid] = 0.f; s_C[c][k][tid] = 0.f; }
        }
        for (int d = d0; d < d1; ++d) {
            const int J = I + d < G.n ? I + d : I + d - G.n;
            const int jb = off + J * SY_T;
            if (d == 0) {
                // ordered pairs inside tile I, self pair skipped; target side only
                for (int sb = 0; sb < SY_T; sb += SY_DTILE) {
                    __syncthreads();
                    for (int l = tid; l < SY_DTILE; l += SY_THREADS) {
                        const int j = jb + sb + l;
                        SrcPk sp;
                        if (j < lim) {
                            const float4 s = L.sources[j];
                            const float kq = kCs * s.w;
                            sp.xx = pk(s.x, s.x); sp.yy = pk(s.y, s.y); sp.zz = pk(s.z, s.z); sp.qq = pk(kq, kq);
                        } else {
                            sp.xx = sp.yy = sp.zz = pk(2e18f, 2e18f);
                            sp.qq = pk(0.f, 0.f);
                        }
                        s_src[l] = sp;
                    }
                    __syncthreads();
                    float part[SY_NI][4];
#pragma unroll
                    for (int k = 0; k < SY_NI; ++k) part[k][0] = part[k][1] = part[k][2] = part[k][3] = 0.f;
                    for (int jj = 0; jj < SY_DTILE; ++jj) {
                        const int j = jb + sb + jj;
                        float sx, sy, sz, sq, dum;
                        upk(s_src[jj].xx, sx, dum); upk(s_src[jj].yy, sy, dum);
                        upk(s_src[jj].zz, sz, dum); upk(s_src[jj].qq, sq, dum);
#pragma unroll
                        for (int k = 0; k < SY_NI; ++k) {
                            const int i = base + k * SY_THREADS + tid;
                            if (j == i) continue;
                            float txk, tyk, tzk, t2;
                            if (k & 1) { upk(TX[k >> 1], t2, txk); upk(TY[k >> 1], t2, tyk); upk(TZ[k >> 1], t2, tzk); }
                            else { upk(TX[k >> 1], txk, t2); upk(TY[k >> 1], tyk, t2); upk(TZ[k >> 1], tzk, t2); }
                            const float dx = __fsub_rn(txk, sx), dy = __fsub_rn(tyk, sy), dz = __fsub_rn(tzk, sz);
                            const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, L.eps2)));
                            const float inv = rsq(r2);
                            const float s = sq * inv;
                            const float s3 = s * (inv * inv);
                            part[k][0] = fmaf(dx, s3, part[k][0]);
                            part[k][1] = fmaf(dy, s3, part[k][1]);
                            part[k][2] = fmaf(dz, s3, part[k][2]);
                            part[k][3] += s;
                        }
                    }
                    if (WANT_V) {
#pragma unroll
                        for (int k = 0; k < SY_NI; ++k) part[k][3] *= SY_VS;
                    }
#pragma unroll
                    for (int k = 0; k < SY_NI; ++k)
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            float sv = s_S[c][k][tid], cv = s_C[c][k][tid];
                            two_sum_acc(sv, cv, part[k][c]);
                            s_S[c][k][tid] = sv;
                            s_C[c][k][tid] = cv;
                        }
                }
                continue;
            }
            // off-diagonal item: source-side sums of tile J, compensated, in shared memory
            __syncthreads();
            for (int l = tid; l < 2 * NC * SY_T; l += SY_THREADS) s_jS[l] = 0.f;   // s_jS and s_jC
            __syncthreads();
            u64 AX[SY_NP], AY[SY_NP], AZ[SY_NP], AV[SY_NP];
#pragma unroll
            for (int p = 0; p < SY_NP; ++p) AX[p] = AY[p] = AZ[p] = AV[p] = 0ull;
            // one charge value in each tile: k_C q factored out of the loop
            const float qJ = tileq[off / SY_T + J], qI = tileq[off / SY_T + I];
            const bool uni = qJ == qJ && qI == qI;
            // factors applied once per sum: k_C q of the tile (field) when the charge
            // is factored out, and the potential's 2^-40
            const float afac = uni ? kCs * qJ : 1.f, pfac = uni ? kCs * qI : 1.f;
            const float afac_v = uni ? (kCs * qJ) * SY_VS : SY_VS, pfac_v = uni ? (kCs * qI) * SY_VS : SY_VS;
            auto rounds = [&](auto uni_c) {
            constexpr bool UNI = decltype(uni_c)::value;
            for (int r = 0; r < SY_NG; ++r) {
                const int grp = (r + (SY_NG / SY_WARPS) * warp) % SY_NG;   // distinct per warp in a round
                const int j0 = jb + grp * 32;
                float4 sj = j0 + lane < lim ? L.sources[j0 + lane] : make_float4(2e18f, 2e18f, 2e18f, 0.f);
                float jx = sj.x, jy = sj.y, jz = sj.z, jq = UNI ? 0.f : kCs * sj.w;
                // the source's reaction sums travel with it as f32x2 packs (the two
                // halves are added once it is back): the FMAs accumulate into them
                u64 PX = 0ull, PY = 0ull, PZ = 0ull, PV = 0ull;
                for (int s = 0; s < 32; ++s) {
                    const u64 JX = pk(jx, jx), JY = pk(jy, jy), JZ = pk(jz, jz), JQ = pk(jq, jq);
#pragma unroll
                    for (int p = 0; p < SY_NP; ++p) {
                        const u64 dx = sub2(TX[p], JX);
                        const u64 dy = sub2(TY[p], JY);
                        const u64 dz = sub2(TZ[p], JZ);
                        u64 r2 = fma2(dx, dx, EPS2);
                        r2 = fma2(dy, dy, r2);
                        r2 = fma2(dz, dz, r2);
                        float ra, rb;
                        upk(r2, ra, rb);
                        const u64 inv = pk(rsq(ra), rsq(rb));
                        const u64 inv3 = mul2(mul2(inv, inv), inv);
                        const u64 si = UNI ? inv3 : mul2(JQ, inv3);
                        const u64 sjp = UNI ? inv3 : mul2(QI[p], inv3);
                        AX[p] = fma2(dx, si, AX[p]);
                        AY[p] = fma2(dy, si, AY[p]);
                        AZ[p] = fma2(dz, si, AZ[p]);
                        PX = fma2(dx, sjp, PX);
                        PY = fma2(dy, sjp, PY);
                        PZ = fma2(dz, sjp, PZ);
                        if (WANT_V) {
                            AV[p] = UNI ? add2(AV[p], inv) : fma2(JQ, inv, AV[p]);
                            PV = UNI ? add2(PV, inv) : fma2(QI[p], inv, PV);
                        }
                    }
                    // pass the source and its sums to the next lane
                    const int src = (lane + 1) & 31;
                    jx = __shfl_sync(0xffffffffu, jx, src);
                    jy = __shfl_sync(0xffffffffu, jy, src);
                    jz = __shfl_sync(0xffffffffu, jz, src);
                    if (!UNI) jq = __shfl_sync(0xffffffffu, jq, src);
                    PX = __shfl_sync(0xffffffffu, PX, src);
                    PY = __shfl_sync(0xffffffffu, PY, src);
                    PZ = __shfl_sync(0xffffffffu, PZ, src);
                    if (WANT_V) PV = __shfl_sync(0xffffffffu, PV, src);
                }
                float ax, ay, az, av = 0.f;
                {
                    float a, b;
                    upk(PX, a, b); ax = a + b;
                    upk(PY, a, b); ay = a + b;
                    upk(PZ, a, b); az = a + b;
                    if (WANT_V) { upk(PV, a, b); av = a + b; }
                }
                if (UNI) { ax *= pfac; ay *= pfac; az *= pfac; }
                if (WANT_V) av *= pfac_v;
                // after 32 passes the sums are back with their source: add this warp's part
                {
                    const int jl = grp * 32 + lane;
                    float sv, cv;
                    sv = s_jS[0 * SY_T + jl]; cv = s_jC[0 * SY_T + jl]; two_sum_acc(sv, cv, ax);
                    s_jS[0 * SY_T + jl] = sv; s_jC[0 * SY_T + jl] = cv;
                    sv = s_jS[1 * SY_T + jl]; cv = s_jC[1 * SY_T + jl]; two_sum_acc(sv, cv, ay);
                    s_jS[1 * SY_T + jl] = sv; s_jC[1 * SY_T + jl] = cv;
                    sv = s_jS[2 * SY_T + jl]; cv = s_jC[2 * SY_T + jl]; two_sum_acc(sv, cv, az);
                    s_jS[2 * SY_T + jl] = sv; s_jC[2 * SY_T + jl] = cv;
                    if (WANT_V) {
                        sv = s_jS[3 * SY_T + jl]; cv = s_jC[3 * SY_T + jl]; two_sum_acc(sv, cv, av);
                        s_jS[3 * SY_T + jl] = sv; s_jC[3 * SY_T + jl] = cv;
                    }
                }
                if ((r + 1) % SY_FOLD == 0) {
#pragma unroll
                    for (int p = 0; p < SY_NP; ++p) {
                        float a, b;
                        float sv, cv;
#define SY_FOLD1(Acc, c)                                                                   \
    upk(Acc[p], a, b);                                                                     \
    if (c == NC - 1 && WANT_V) { a *= afac_v; b *= afac_v; }                               \
    else if (UNI) { a *= afac; b *= afac; }                                                \
    sv = s_S[c][2 * p][tid]; cv = s_C[c][2 * p][tid]; two_sum_acc(sv, cv, a);              \
    s_S[c][2 * p][tid] = sv; s_C[c][2 * p][tid] = cv;                                      \
    sv = s_S[c][2 * p + 1][tid]; cv = s_C[c][2 * p + 1][tid]; two_sum_acc(sv, cv, b);      \
    s_S[c][2 * p + 1][tid] = sv; s_C[c][2 * p + 1][tid] = cv;                              \
    Acc[p] = 0ull;
                        SY_FOLD1(AX, 0)
                        SY_FOLD1(AY, 1)
                        SY_FOLD1(AZ, 2)
                        if (WANT_V) { SY_FOLD1(AV, NC - 1) }
#undef SY_FOLD1
                    }
                }
                __syncthreads();
            }
            };
            if (uni) rounds(SyBool<true>{});
            else rounds(SyBool<false>{});
            // the item's source-side sums (S + C) to its own slot
            float *jp = jpart + (BATCH ? s_joff : 0) + ((size_t)I * jd + (d - klo * CH)) * 4 * SY_T;
            for (int l = tid; l < NC * SY_T; l += SY_THREADS) jp[l] = s_jS[l] + s_jC[l];
        }
        // the unit's target-side sums (S and C) to its own slot
        float *ip = ipart + (BATCH ? s_ioff : 0) + ((size_t)I * kn + (kch - klo)) * 8 * SY_T;
#pragma unroll
        for (int k = 0; k < SY_NI; ++k)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                ip[(2 * c) * SY_T + k * SY_THREADS + tid] = s_S[c][k][tid];
                ip[(2 * c + 1) * SY_T + k * SY_THREADS + tid] = s_C[c][k][tid];
            }
    }
}

// E_out[t] = init + target-side sums of t's row + minus the source-side sums of
// every item whose second tile holds t, added in a fixed order (FP64).  t is a
// slot of the sorted copy; perm[t] the charge it holds.
template <bool WANT_V, int CH = SY_CH>
__global__ void nbsym_fold_kernel(FieldLaunch L, const float *jpart, const float *ipart, int add, const int32_t *perm,
                                  SymBatch SB, SymPass PS)
{
    constexpr int NC = WANT_V ? 4 : 3;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int nt, off = 0;
    long long joff = 0, ioff = 0;
    if (SB.nb) {
        if (t >= SB.seg_off[SB.nb]) return;
        const int c = SB.slot_cham[t / OBEM_SEG_ALIGN];
        off = SB.seg_off[c];
        nt = SB.n[c];
        joff = SB.joff[c];
        ioff = SB.ioff[c];
    } else {
        nt = L.nt_dev ? *L.nt_dev : L.nt;
    }
    const int lt = t - off;
    if (lt >= nt) return;
    const SymGeom G = sym_geom_ch<CH>(nt);
    const int T = lt / SY_T, w = lt % SY_T;
    const int o = perm ? perm[t] : t;                  // sorted slot t is charge o
    // this pass's units and diagonals (all of them for a batch)
    const int kn = PS.kch_n ? min(PS.kch_n, G.nch - PS.kch_lo) : G.nch;
    const int klo = PS.kch_n ? PS.kch_lo : 0;
    const int jd = PS.kch_n ? PS.jd : G.hmax + 1;
    const int dlo = max(1, klo * CH), dhi = min(G.hmax, klo * CH + jd - 1);
    double e[4] = {0.0, 0.0, 0.0, 0.0};
    if (!PS.first) {
        const double *a = PS.acc + 4 * (size_t)t;
        e[0] = a[0]; e[1] = a[1]; e[2] = a[2]; e[3] = a[3];
    } else if (add) {
        const float4 q = L.E_out[o];
        e[0] = q.x; e[1] = q.y; e[2] = q.z; e[3] = q.w;
    } else {
        e[0] = L.e_ext.x; e[1] = L.e_ext.y; e[2] = L.e_ext.z;
    }
    for (int k = 0; k < kn; ++k) {
        const float *ip = ipart + ioff + ((size_t)T * kn + k) * 8 * SY_T;
#pragma unroll
        for (int c = 0; c < NC; ++c) e[c] += (double)ip[(2 * c) * SY_T + w] + (double)ip[(2 * c + 1) * SY_T + w];
    }
    // the items (I, d) with I + d = T (mod n): four loads in flight per round,
    // added in order into compensated binary32 sums (TwoSum: ~2^-48 relative,
    // like FP64, on the FP32 pipe; GB300's FP64 pipe would take ~5 ms here)
    constexpr int FU = 4;
    float js[NC], jc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { js[c] = 0.f; jc[c] = 0.f; }
    for (int d0 = dlo; d0 <= dhi; d0 += FU) {
        float v[FU][NC];
#pragma unroll
        for (int u = 0; u < FU; ++u) {
            const int d = d0 + u;
            const int I = T - d >= 0 ? T - d : T - d + G.n;
            const bool ok = d <= dhi && d <= sym_h(G, I);
            const float *jp = jpart + joff + ((size_t)I * jd + (ok ? d - klo * CH : 0)) * 4 * SY_T;
#pragma unroll
            for (int c = 0; c < NC; ++c) v[u][c] = ok ? jp[c * SY_T + w] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < FU; ++u)
#pragma unroll
            for (int c = 0; c < NC; ++c) two_sum_acc(js[c], jc[c], c < 3 ? -v[u][c] : v[u][c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) e[c] += (double)js[c] + (double)jc[c];
    if (PS.last) {
        L.E_out[o] = make_float4((float)e[0], (float)e[1], (float)e[2], WANT_V ? (float)e[3] : 0.f);
    } else {
        double *a = PS.acc + 4 * (size_t)t;
        a[0] = e[0]; a[1] = e[1]; a[2] = e[2]; a[3] = e[3];
    }
}

// occupancy-limited persistent grid of the symmetric kernel
int obem_sym_grid(int device)
{
    int sms = 0, best = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    void (*ks[])(FieldLaunch, float *, float *, int *, const float *, SymBatch, SymPass) = {
        nbsym_kernel<true, false>, nbsym_kernel<false, false>, nbsym_kernel<false, true>,
        nbsym_kernel<true, false, SY_CH_SMALL>, nbsym_kernel<false, false, SY_CH_SMALL>,
        nbsym_kernel<true, false, SY_CH_MID>, nbsym_kernel<false, false, SY_CH_MID>};
    const size_t sm[] = {sym_smem(4), sym_smem(3), sym_smem(3), sym_smem(4), sym_smem(3), sym_smem(4), sym_smem(3)};
    for (int q = 0; q < 7; ++q) {
        if (cudaFuncSetAttribute(ks[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[q]) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ks[q], SY_THREADS, sm[q]) != cudaSuccess) return 0;
        best = (best == 0 || occ < best) ? occ : best;
    }
    return sms * (best > 0 ? best : 1);
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
    const bool add = cells || L.add_init;      // E_out holds a field the all-pairs sum adds to
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
            block_list_kernel<<<1, 1024, 0, s>>>(ctx->s_hist, L.nt, L.nt_dev, (int2 *)L.blocks, (int32_t *)L.nblocks);
            binsort(ctx->s_code, ctx->s_code, (int32_t *)L.perm, ctx->s_tk, ctx->s_tv, ctx->s_rh, L.nt, L.nt_dev,
                    capacity_targets, s);
            OBEM_LAUNCH(ctx);
            if (L.events) ctx->launches += 12;
        }
        const int nsuper = capacity_targets < OBEM_NSUPER ? capacity_targets : OBEM_NSUPER;
        dim3 cgrid((capacity_targets + CT_BLOCK - 1) / CT_BLOCK + (L.blocks ? nsuper : 0));
        if (L.events) cudaEventRecord(L.events[4], s);
        if (L.want_v) {
            if (L.counters) { near_closed_kernel<true, true><<<cgrid, CT_THREADS, 0, s>>>(L); near_quad_kernel<true, true><<<cgrid, CT_THREADS, 0, s>>>(L); }
            else { near_closed_kernel<true, false><<<cgrid, CT_THREADS, 0, s>>>(L); near_quad_kernel<true, false><<<cgrid, CT_THREADS, 0, s>>>(L); }
        } else {
            if (L.counters) { near_closed_kernel<false, true><<<cgrid, CT_THREADS, 0, s>>>(L); near_quad_kernel<false, true><<<cgrid, CT_THREADS, 0, s>>>(L); }
            else { near_closed_kernel<false, false><<<cgrid, CT_THREADS, 0, s>>>(L); near_quad_kernel<false, false><<<cgrid, CT_THREADS, 0, s>>>(L); }
        }
        if (L.events) cudaEventRecord(L.events[5], s);
        // far cells in groups: the context's own cells, one set of targets
        const bool grouped = ctx->ngrp > 0 && L.panels.c_a == ctx->d_c_a && !L.block_cham;
        if (grouped) {
            CellGroups G;
            int fitted = 0;
            int rc = obem_cell_groups_fit(ctx, L.sigma, s, &G, &fitted);
            if (rc != OBEM_OK) return rc;
            if (L.events) ctx->launches += fitted;
            if (L.want_v) {
                if (L.counters) cell_group_kernel<true, true><<<cgrid, CT_THREADS, 0, s>>>(L, G);
                else cell_group_kernel<true, false><<<cgrid, CT_THREADS, 0, s>>>(L, G);
            } else {
                if (L.counters) cell_group_kernel<false, true><<<cgrid, CT_THREADS, 0, s>>>(L, G);
                else cell_group_kernel<false, false><<<cgrid, CT_THREADS, 0, s>>>(L, G);
            }
        } else if (L.want_v) {
            if (L.counters) cell_kernel<true, true><<<cgrid, CT_THREADS, 0, s>>>(L);
            else cell_kernel<true, false><<<cgrid, CT_THREADS, 0, s>>>(L);
        } else {
            if (L.counters) cell_kernel<false, true><<<cgrid, CT_THREADS, 0, s>>>(L);
            else cell_kernel<false, false><<<cgrid, CT_THREADS, 0, s>>>(L);
        }
        OBEM_LAUNCH(ctx);
        if (L.events) ctx->launches += 3;
    }
    if (L.events) cudaEventRecord(L.events[1], s);
    if (charges) {
        if (L.counters) {
            pair_count_kernel<<<1, 32, 0, s>>>(L);
            OBEM_LAUNCH(ctx);
            if (L.events) ctx->launches++;
        }
        // self_exclude: the targets are the sources (same charges, nt == ns)
        const bool nn = L.nn_grid > 0 && L.self_exclude && !L.shard;
        const bool sym = !nn && ctx->sym_jpart && L.self_exclude && !L.shard && capacity_targets <= ctx->sym_cap;
        if (nn) {
            int rc = obem_launch_nbody_nn(ctx, L.sources, L.nt_dev, capacity_targets, L.nn_grid, L.eps2, L.E_out,
                                          L.e_ext, add ? 1 : 0, s);
            if (rc != OBEM_OK) return rc;
            if (L.events) ctx->launches += 7;
        } else if (sym) {
            // charges ordered by charge value (stable), per-tile common charge
            const int nb = obem_sym_part_blocks(capacity_targets);
            SymBatch SB;
            memset(&SB, 0, sizeof SB);
            sym_part_count_kernel<<<nb, SP_BLOCK, 0, s>>>(L.sources, L.nt, L.nt_dev, SB, ctx->sym_bcnt);
            sym_part_scan_kernel<<<1, 1024, 0, s>>>(ctx->sym_bcnt, nb, SB, ctx->sym_bcnt + nb);
            sym_part_scatter_kernel<<<nb, SP_BLOCK, 0, s>>>(L.targets, L.sources, L.nt, L.nt_dev, SB, ctx->sym_bcnt,
                                                           ctx->sym_bcnt + nb, ctx->sym_sorted, ctx->sym_perm);
            sym_tileq_kernel<<<obem_sym_tiles(capacity_targets), 256, 0, s>>>(ctx->sym_sorted, L.nt, L.nt_dev, SB,
                                                                             ctx->sym_tileq);
            OBEM_LAUNCH(ctx);
            FieldLaunch Ls = L;
            Ls.targets = ctx->sym_sorted;
            Ls.sources = ctx->sym_sorted;
            Ls.eps2 = L.eps2 * SY_QS;                    // the sorted copy's positions are x 2^40
            // the diagonals in passes of SY_PASS_CH units per row, each folded
            // in order into a per-charge FP64 accumulator: partial sums O(N)
            // (a fixed pass size keeps the summation order, and so the bits,
            // independent of the memory available)
            // contexts for at most SY_SMALL_TILES / SY_MID_TILES tiles take
            // units of fewer items, so that a set's few tile pairs still
            // spread over the SMs (separate instantiations: the large-set
            // kernel is untouched); chosen by the capacity the partial-sum
            // scratch was sized for (the live count is on the device)
            const int ntile = sym_geom(ctx->sym_cap).n;
            const int ch = ntile <= SY_SMALL_TILES ? SY_CH_SMALL : (ntile <= SY_MID_TILES ? SY_CH_MID : SY_CH);
            const SymGeom Gc = ch == SY_CH_SMALL ? sym_geom_ch<SY_CH_SMALL>(capacity_targets)
                               : ch == SY_CH_MID ? sym_geom_ch<SY_CH_MID>(capacity_targets) : sym_geom(capacity_targets);
            const int npass = (Gc.nch + SY_PASS_CH - 1) / SY_PASS_CH;
            const dim3 sg(ctx->sym_grid);
            const int fb = (capacity_targets + 255) / 256;
            typedef void (*SymK)(FieldLaunch, float *, float *, int *, const float *, SymBatch, SymPass);
            typedef void (*FoldK)(FieldLaunch, const float *, const float *, int, const int32_t *, SymBatch, SymPass);
            const SymK kern = L.want_v ? (ch == SY_CH_SMALL ? nbsym_kernel<true, false, SY_CH_SMALL>
                                          : ch == SY_CH_MID ? nbsym_kernel<true, false, SY_CH_MID>
                                                            : nbsym_kernel<true, false>)
                                       : (ch == SY_CH_SMALL ? nbsym_kernel<false, false, SY_CH_SMALL>
                                          : ch == SY_CH_MID ? nbsym_kernel<false, false, SY_CH_MID>
                                                            : nbsym_kernel<false, false>);
            const FoldK fold = L.want_v ? (ch == SY_CH_SMALL ? nbsym_fold_kernel<true, SY_CH_SMALL>
                                           : ch == SY_CH_MID ? nbsym_fold_kernel<true, SY_CH_MID>
                                                             : nbsym_fold_kernel<true>)
                                        : (ch == SY_CH_SMALL ? nbsym_fold_kernel<false, SY_CH_SMALL>
                                           : ch == SY_CH_MID ? nbsym_fold_kernel<false, SY_CH_MID>
                                                             : nbsym_fold_kernel<false>);
            const size_t ksmem = sym_smem(L.want_v ? 4 : 3);
            for (int pz = 0; pz < npass; ++pz) {
                SymPass PS;
                PS.kch_lo = pz * SY_PASS_CH;
                PS.kch_n = SY_PASS_CH;
                PS.jd = Gc.hmax + 1 < SY_PASS_CH * ch ? Gc.hmax + 1 : SY_PASS_CH * ch;   // within the allocation
                PS.first = pz == 0;
                PS.last = pz == npass - 1;
                PS.acc = ctx->sym_acc;
                OBEM_CUDA(ctx, cudaMemsetAsync(ctx->sym_counter, 0, sizeof(int), s));
                kern<<<sg, SY_THREADS, ksmem, s>>>(Ls, ctx->sym_jpart, ctx->sym_ipart, ctx->sym_counter, ctx->sym_tileq,
                                                   SB, PS);
                OBEM_LAUNCH(ctx);
                fold<<<fb, 256, 0, s>>>(L, ctx->sym_jpart, ctx->sym_ipart, add ? 1 : 0, ctx->sym_perm, SB, PS);
                OBEM_LAUNCH(ctx);
            }
            if (L.events) ctx->launches += 4 + 2 * npass;
        } else if (L.want_v) {
            if (add) nbody_kernel<true, true><<<grid, FT_THREADS, 0, s>>>(L);
            else nbody_kernel<true, false><<<grid, FT_THREADS, 0, s>>>(L);
        } else {
            if (add) nbody_kernel<false, true><<<grid, FT_THREADS, 0, s>>>(L);
            else nbody_kernel<false, false><<<grid, FT_THREADS, 0, s>>>(L);
        }
        if (!sym && !nn) {
            OBEM_LAUNCH(ctx);
            if (L.events) ctx->launches++;
        }
    }
    if (!cells && !charges && !L.add_init) {
        const_field_kernel<<<(capacity_targets + 255) / 256, 256, 0, s>>>(L);
        OBEM_LAUNCH(ctx);
        if (L.events) ctx->launches++;
    }
    if (L.events) cudaEventRecord(L.events[2], s);
    return OBEM_OK;
}

// ====================================================================
// Batch of chambers.

size_t obem_sym_sizes(int capacity, size_t *ipart_floats)
{
    *ipart_floats = obem_sym_ipart_floats(capacity);
    return obem_sym_jpart_floats(capacity);
}

// cell-kernel blocks of every chamber: ceil(n[c] / cut) blocks of consecutive
// live slots each (one block of 1024 threads)
__global__ void bt_blocks_kernel(FieldBatch F, int2 *blocks, int32_t *block_cham, int32_t *nblocks)
{
    __shared__ int32_t part[1024];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < F.nb; c0 += 1024) {
        const int c = c0 + threadIdx.x;
        const int n = c < F.nb ? F.sym.n[c] : 0;
        const int k = (n + F.cut - 1) / F.cut;
        part[threadIdx.x] = k;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        int b = carry + part[threadIdx.x] - k;
        const int off = c < F.nb ? F.sym.seg_off[c] : 0;
        for (int q = 0; q < k; ++q, ++b) {
            blocks[b] = make_int2(off + q * F.cut, min(F.cut, n - q * F.cut));
            block_cham[b] = c;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *nblocks = carry;
}

__global__ void bt_const_field_kernel(FieldBatch F, float4 *E_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.slots) return;
    const int c = F.sym.slot_cham[i / OBEM_SEG_ALIGN];
    if (i - F.sym.seg_off[c] >= F.sym.n[c]) return;
    E_out[i] = make_float4(F.e_ext.x, F.e_ext.y, F.e_ext.z, 0.f);
}

int obem_launch_field_batch(obem_ctx *ctx, const FieldBatch &F, const float4 *pos_q, float4 *E_out, cudaStream_t s)
{
    if (F.cut < 32 || F.cut > CT_BLOCK) return obem_fail(ctx, OBEM_ERR_ARG, "batch: cell block size outside 32..512");
    FieldLaunch L;
    memset(&L, 0, sizeof L);
    L.targets = pos_q;
    L.nt = F.slots;
    L.sources = pos_q;
    L.self_exclude = 1;
    L.eps2 = F.eps2;
    L.E_out = E_out;
    L.e_ext = F.e_ext;
    L.want_v = 0;
    if (F.cells) {
        L.sigma = F.sigma;
        L.panels = F.panels;
        L.blocks = F.blocks;
        L.nblocks = F.nblocks;
        L.block_cham = F.block_cham;
        L.cham_pan = F.cham_pan;
        bt_blocks_kernel<<<1, 1024, 0, s>>>(F, F.blocks, F.block_cham, F.nblocks);
        OBEM_LAUNCH(ctx);
        const dim3 cg(F.max_blocks);
        near_closed_kernel<false, false><<<cg, CT_THREADS, 0, s>>>(L);
        near_quad_kernel<false, false><<<cg, CT_THREADS, 0, s>>>(L);
        cell_kernel<false, false, true><<<cg, CT_THREADS, 0, s>>>(L);
        OBEM_LAUNCH(ctx);
    }
    if (F.charges) {
        const int nsb = F.slots / SP_BLOCK;
        sym_part_count_kernel<<<nsb, SP_BLOCK, 0, s>>>(pos_q, 0, NULL, F.sym, F.bcnt);
        sym_part_scan_kernel<<<F.nb, 1024, 0, s>>>(F.bcnt, 0, F.sym, F.sym.negtot);
        sym_part_scatter_kernel<<<nsb, SP_BLOCK, 0, s>>>(pos_q, pos_q, 0, NULL, F.sym, F.bcnt, F.sym.negtot, F.sorted,
                                                        F.perm);
        sym_tileq_kernel<<<nsb, 256, 0, s>>>(F.sorted, 0, NULL, F.sym, F.tileq);
        sym_units_kernel<<<1, 1024, 0, s>>>(F.sym);
        OBEM_LAUNCH(ctx);
        FieldLaunch Ls = L;
        Ls.targets = F.sorted;
        Ls.sources = F.sorted;
        Ls.eps2 = L.eps2 * SY_QS;                        // the sorted copy's positions are x 2^40
        OBEM_CUDA(ctx, cudaMemsetAsync(F.counter, 0, sizeof(int), s));
        nbsym_kernel<false, true><<<F.sym_grid, SY_THREADS, sym_smem(3), s>>>(Ls, F.jpart, F.ipart, F.counter, F.tileq,
                                                                       F.sym, SymPass{0, 0, 0, 1, 1, NULL});
        OBEM_LAUNCH(ctx);
        nbsym_fold_kernel<false><<<F.slots / 256, 256, 0, s>>>(L, F.jpart, F.ipart, F.cells ? 1 : 0, F.perm, F.sym,
                                                               SymPass{0, 0, 0, 1, 1, NULL});
        OBEM_LAUNCH(ctx);
    }
    if (!F.cells && !F.charges) {
        bt_const_field_kernel<<<F.slots / 256, 256, 0, s>>>(F, E_out);
        OBEM_LAUNCH(ctx);
    }
    return OBEM_OK;
}

// ====================================================================
// Field evaluation with no context and no allocation.
//
// For callers that cannot call cudaMalloc -- plug-ins that must live inside a
// host application's fixed device-memory budget, or real-time loops where
// the latency or failure of an allocation is not allowed -- and that
// therefore cannot create an obem_ctx (whose creation and mesh upload
// allocate).  The same kernels as obem_field_eval run on
// scratch held in one file-scope device array of fixed size, reached through
// cudaGetSymbolAddress.
// ====================================================================
#define NA_MAX_TARGETS OBEM_NOALLOC_MAX_TARGETS
#define NA_MAX_CELLS OBEM_NOALLOC_MAX_CELLS

namespace {
constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_CELLS_BYTES = na_align(sizeof(float4) * 6 * (size_t)NA_MAX_CELLS);
constexpr size_t NA_CODE_BYTES = na_align(sizeof(uint32_t) * (size_t)NA_MAX_TARGETS);
constexpr size_t NA_PERM_BYTES = na_align(sizeof(int32_t) * (size_t)NA_MAX_TARGETS);
constexpr size_t NA_HIST_BYTES = na_align(sizeof(int32_t) * (size_t)OBEM_NBINS);
constexpr size_t NA_NBLK = (size_t)NA_MAX_TARGETS / 512 + 2 + OBEM_NSUPER;
constexpr size_t NA_BLOCKS_BYTES = na_align(sizeof(int2) * NA_NBLK);
constexpr size_t NA_MISC_BYTES = 256;   // number of blocks, bounding box
constexpr size_t NA_TK_BYTES = na_align(sizeof(uint32_t) * (size_t)NA_MAX_TARGETS);    // bin sort scratch
constexpr size_t NA_TV_BYTES = na_align(sizeof(int32_t) * (size_t)NA_MAX_TARGETS);
constexpr size_t NA_RH_BYTES = na_align(sizeof(int32_t) * (64 * ((size_t)NA_MAX_TARGETS / 1024 + 1) + 1));
constexpr size_t NA_BYTES = NA_CELLS_BYTES + NA_CODE_BYTES + NA_PERM_BYTES + NA_HIST_BYTES + NA_BLOCKS_BYTES +
                            NA_MISC_BYTES + NA_TK_BYTES + NA_TV_BYTES + NA_RH_BYTES;
}  // namespace

// The scratch of obem_field_eval_noalloc (about 5 MB); every GPU that loads
// the library holds it until the process exits.
static __device__ __align__(256) unsigned char na_scratch[NA_BYTES];

// Device address of na_scratch, per device ordinal (set on the first call
// made with that device current).
#define NA_MAX_DEVICES 64
static unsigned char *na_base[NA_MAX_DEVICES];

// Derived cell geometry (the layout of PanelsDev) from FP64 vertices.
__global__ void na_cells_kernel(const double *v64, int np, float4 *c_a, float4 *g0_h, float4 *g1, float4 *g2,
                                float4 *nrm, float4 *c_lo)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double *v = v64 + 9 * (size_t)i;
    double cc[3], e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        cc[k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0;
        e1[k] = v[3 + k] - v[k];
        e2[k] = v[6 + k] - v[k];
    }
    double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2], nz = e1[0] * e2[1] - e1[1] * e2[0];
    double a2 = sqrt(nx * nx + ny * ny + nz * nz);
    double h2 = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *a = v + 3 * e, *b = v + 3 * ((e + 1) % 3);
        double d = (a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]);
        h2 = d > h2 ? d : h2;
    }
    float4 ca = make_float4((float)cc[0], (float)cc[1], (float)cc[2], (float)(OBEM_KC * 0.5 * a2));
    c_a[i] = ca;
    g0_h[i] = make_float4((float)(v[0] - cc[0]), (float)(v[1] - cc[1]), (float)(v[2] - cc[2]), (float)h2);
    g1[i] = make_float4((float)(v[3] - cc[0]), (float)(v[4] - cc[1]), (float)(v[5] - cc[2]), 0.f);
    g2[i] = make_float4((float)(v[6] - cc[0]), (float)(v[7] - cc[1]), (float)(v[8] - cc[2]), 0.f);
    nrm[i] = make_float4((float)(nx / a2), (float)(ny / a2), (float)(nz / a2), 0.f);
    c_lo[i] = make_float4((float)(cc[0] - (double)ca.x), (float)(cc[1] - (double)ca.y),
                          (float)(cc[2] - (double)ca.z), 0.f);
}

// bounding box of the vertices, one block; box = [lo.xyz, hi.xyz]
__global__ void na_bbox_kernel(const double *v64, int np, float *box)
{
    __shared__ float red[6][32];
    float mn[3] = {3e38f, 3e38f, 3e38f}, mx[3] = {-3e38f, -3e38f, -3e38f};
    for (int q = threadIdx.x; q < 3 * np; q += blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            float x = (float)v64[3 * (size_t)q + k];
            mn[k] = fminf(mn[k], x);
            mx[k] = fmaxf(mx[k], x);
        }
    }
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o; o >>= 1) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k) { red[k][threadIdx.x >> 5] = mn[k]; red[3 + k][threadIdx.x >> 5] = mx[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) {
            float v = red[k][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = k < 3 ? fminf(v, red[k][w]) : fmaxf(v, red[k][w]);
            box[k] = v;
        }
    }
}

// binning with the grid read from device memory (box from na_bbox_kernel)
__global__ void na_bin_count_kernel(FieldLaunch L, const float *box, uint32_t *code, int32_t *hist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.nt) return;
    const float3 lo = make_float3(box[0], box[1], box[2]);
    const float3 sc = make_float3((float)OBEM_BINS_PER_AXIS / fmaxf(box[3] - box[0], 1e-30f),
                                  (float)OBEM_BINS_PER_AXIS / fmaxf(box[4] - box[1], 1e-30f),
                                  (float)OBEM_BINS_PER_AXIS / fmaxf(box[5] - box[2], 1e-30f));
    float4 p = L.targets[i];
    int ix = (int)fminf(fmaxf((p.x - lo.x) * sc.x, 0.f), (float)(OBEM_BINS_PER_AXIS - 1));
    int iy = (int)fminf(fmaxf((p.y - lo.y) * sc.y, 0.f), (float)(OBEM_BINS_PER_AXIS - 1));
    int iz = (int)fminf(fmaxf((p.z - lo.z) * sc.z, 0.f), (float)(OBEM_BINS_PER_AXIS - 1));
    uint32_t c = spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
    code[i] = c;
    atomicAdd(&hist[c], 1);
}

static int na_fail(char *err, int32_t err_len, int code, const char *msg)
{
    if (err && err_len > 0) {
        strncpy(err, msg, (size_t)err_len - 1);
        err[err_len - 1] = '\0';
    }
    return code;
}

extern "C" int obem_field_eval_noalloc(const float *targets, int32_t nt, const float *sources, int32_t ns,
                                       int32_t self_exclude, const double *cell_xyz, const float *sigma,
                                       int32_t np, float *E_out, char *err, int32_t err_len,
                                       obem_stream stream)
{
    char msg[256];
    if (nt < 0 || ns < 0 || np < 0) return na_fail(err, err_len, OBEM_ERR_ARG, "negative count");
    if (nt > NA_MAX_TARGETS) {
        snprintf(msg, sizeof msg, "nt = %d exceeds the fixed scratch of %d targets", nt, NA_MAX_TARGETS);
        return na_fail(err, err_len, OBEM_ERR_ARG, msg);
    }
    if (np > NA_MAX_CELLS) {
        snprintf(msg, sizeof msg, "np = %d exceeds the fixed scratch of %d cells", np, NA_MAX_CELLS);
        return na_fail(err, err_len, OBEM_ERR_ARG, msg);
    }
    if (nt == 0) return OBEM_OK;
    if (!targets || !E_out) return na_fail(err, err_len, OBEM_ERR_ARG, "null targets or E_out");
    if (np > 0 && (!cell_xyz || !sigma)) return na_fail(err, err_len, OBEM_ERR_ARG, "cells without vertices or sigma");
    if (self_exclude && (!sources || ns != nt))
        return na_fail(err, err_len, OBEM_ERR_ARG, "self_exclude needs sources with ns == nt");
    if (((uintptr_t)targets | (uintptr_t)E_out | (uintptr_t)sources) & 15)
        return na_fail(err, err_len, OBEM_ERR_ARG, "arrays must be 16-byte aligned");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
        return na_fail(err, err_len, OBEM_ERR_CUDA, "no usable current device");
    if (!na_base[dev]) {
        void *p = NULL;
        cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess) {
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return na_fail(err, err_len, OBEM_ERR_CUDA, msg);
        }
        na_base[dev] = (unsigned char *)p;
    }
    unsigned char *b = na_base[dev];
    float4 *cells = (float4 *)b;
    uint32_t *code = (uint32_t *)(b + NA_CELLS_BYTES);
    int32_t *perm = (int32_t *)(b + NA_CELLS_BYTES + NA_CODE_BYTES);
    int32_t *hist = (int32_t *)(b + NA_CELLS_BYTES + NA_CODE_BYTES + NA_PERM_BYTES);
    int2 *blocks = (int2 *)(b + NA_CELLS_BYTES + NA_CODE_BYTES + NA_PERM_BYTES + NA_HIST_BYTES);
    int32_t *nblocks = (int32_t *)(b + NA_CELLS_BYTES + NA_CODE_BYTES + NA_PERM_BYTES + NA_HIST_BYTES + NA_BLOCKS_BYTES);
    unsigned char *b2 = b + NA_CELLS_BYTES + NA_CODE_BYTES + NA_PERM_BYTES + NA_HIST_BYTES + NA_BLOCKS_BYTES +
                        NA_MISC_BYTES;
    uint32_t *na_tk = (uint32_t *)b2;
    int32_t *na_tv = (int32_t *)(b2 + NA_TK_BYTES);
    int32_t *na_rh = (int32_t *)(b2 + NA_TK_BYTES + NA_TV_BYTES);
    float *box = (float *)(nblocks + 16);
    cudaStream_t s = (cudaStream_t)stream;

    FieldLaunch L;
    memset(&L, 0, sizeof L);
    L.targets = (const float4 *)targets;
    L.nt = nt;
    L.sources = (sources && ns > 0) ? (const float4 *)sources : NULL;
    L.ns = ns;
    L.self_exclude = self_exclude ? 1 : 0;
    L.E_out = (float4 *)E_out;
    L.e_ext = make_float3(0.f, 0.f, 0.f);
    L.want_v = 1;
    const bool cells_on = np > 0;
    if (cells_on) {
        L.sigma = sigma;
        L.panels.c_a = cells;
        L.panels.g0_h = cells + NA_MAX_CELLS;
        L.panels.g1 = cells + 2 * NA_MAX_CELLS;
        L.panels.g2 = cells + 3 * NA_MAX_CELLS;
        L.panels.nrm = cells + 4 * NA_MAX_CELLS;
        L.panels.c_lo = cells + 5 * NA_MAX_CELLS;
        L.panels.v64 = cell_xyz;
        L.panels.np = np;
        L.perm = perm;
        L.blocks = blocks;
        L.nblocks = nblocks;
        na_cells_kernel<<<(np + 127) / 128, 128, 0, s>>>(cell_xyz, np, (float4 *)L.panels.c_a, (float4 *)L.panels.g0_h,
                                                        (float4 *)L.panels.g1, (float4 *)L.panels.g2,
                                                        (float4 *)L.panels.nrm, (float4 *)L.panels.c_lo);
        na_bbox_kernel<<<1, 1024, 0, s>>>(cell_xyz, np, box);
        // the array keeps the previous call's contents: the histogram must restart at zero
        if (cudaMemsetAsync(hist, 0, sizeof(int32_t) * OBEM_NBINS, s) != cudaSuccess)
            return na_fail(err, err_len, OBEM_ERR_CUDA, "cudaMemsetAsync of the histogram failed");
        const int nb = (nt + 255) / 256;
        na_bin_count_kernel<<<nb, 256, 0, s>>>(L, box, code, hist);
        bin_scan_kernel<<<1, 1024, 0, s>>>(hist);
        block_list_kernel<<<1, 1024, 0, s>>>(hist, nt, NULL, blocks, nblocks);
        binsort(code, code, perm, na_tk, na_tv, na_rh, nt, NULL, nt, s);
        const int nsuper = nt < OBEM_NSUPER ? nt : OBEM_NSUPER;
        dim3 cgrid((nt + CT_BLOCK - 1) / CT_BLOCK + nsuper);
        near_closed_kernel<true, false><<<cgrid, CT_THREADS, 0, s>>>(L);
        near_quad_kernel<true, false><<<cgrid, CT_THREADS, 0, s>>>(L);
        cell_kernel<true, false><<<cgrid, CT_THREADS, 0, s>>>(L);
    }
    dim3 grid((nt + FT_BLOCK_TARGETS - 1) / FT_BLOCK_TARGETS);
    if (L.sources) {
        if (cells_on) nbody_kernel<true, true><<<grid, FT_THREADS, 0, s>>>(L);
        else nbody_kernel<true, false><<<grid, FT_THREADS, 0, s>>>(L);
    } else if (!cells_on) {
        const_field_kernel<<<(nt + 255) / 256, 256, 0, s>>>(L);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "kernel launch failed: %s", cudaGetErrorString(e));
        return na_fail(err, err_len, OBEM_ERR_CUDA, msg);
    }
    return OBEM_OK;
}
