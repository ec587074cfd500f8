// Static field map (Sec. 2.4, and the timing set-up of Sec. 2.4's table of
// grid evaluations): the cell field of Eqs. (BEM3), (BEM2) evaluated once on a
// regular grid, then interpolated trilinearly while tracking, instead of being
// summed over every cell at every step (the paper's "static" option; the
// direct sum is its "dynamic" one).
//
// Nodes are generated on the device in bricks of 8 x 8 x 8 = 512 consecutive
// points, so that each brick is one compact block of the cell kernels (no
// spatial sort needed) and the map is stored in brick order; the grid is
// padded to whole bricks (padding nodes continue the grid past hi and are
// never read).
#include "obem_internal.cuh"

#define FM_B 8
#define FM_BRICK (FM_B * FM_B * FM_B)
#define FM_CHUNK (1 << 21)          // nodes evaluated per field launch

__device__ __forceinline__ size_t fm_offset(const FieldMapDev &m, int ix, int iy, int iz)
{
    const int nbx = m.px / FM_B, nby = m.py / FM_B;
    const size_t b = ((size_t)(iz / FM_B) * nby + (iy / FM_B)) * nbx + (ix / FM_B);
    return b * FM_BRICK + ((iz % FM_B) * FM_B + (iy % FM_B)) * FM_B + (ix % FM_B);
}

// positions of the nodes [first, first + count) in brick order
__global__ void fm_nodes_kernel(FieldMapDev m, size_t first, int count, float4 *pts)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const size_t t = first + k;
    const size_t b = t / FM_BRICK;
    const int w = (int)(t % FM_BRICK);
    const int nbx = m.px / FM_B, nby = m.py / FM_B;
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((size_t)nbx * nby));
    const int ix = bx * FM_B + w % FM_B, iy = by * FM_B + (w / FM_B) % FM_B, iz = bz * FM_B + w / (FM_B * FM_B);
    pts[k] = make_float4((float)(m.lo[0] + ix * m.step[0]), (float)(m.lo[1] + iy * m.step[1]),
                         (float)(m.lo[2] + iz * m.step[2]), 0.f);
}

// trilinear interpolation of the map at points (clamped to the grid's box);
// out = interpolated (Ex, Ey, Ez, V) + (e_ext, 0)
__device__ __forceinline__ float4 fm_interp(const FieldMapDev &m, float4 p)
{
    float f[3], t[3];
    int i0[3];
    const float pp[3] = {p.x, p.y, p.z};
    const int n[3] = {m.nx, m.ny, m.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[a] = (float)(((double)pp[a] - m.lo[a]) / m.step[a]);
        f[a] = fminf(fmaxf(f[a], 0.f), (float)(n[a] - 1));
        i0[a] = min((int)floorf(f[a]), n[a] - 2);
        t[a] = f[a] - (float)i0[a];
    }
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        const float w = (dx ? t[0] : 1.f - t[0]) * (dy ? t[1] : 1.f - t[1]) * (dz ? t[2] : 1.f - t[2]);
        const float4 v = m.nodes[fm_offset(m, i0[0] + dx, i0[1] + dy, i0[2] + dz)];
        r.x = fmaf(w, v.x, r.x);
        r.y = fmaf(w, v.y, r.y);
        r.z = fmaf(w, v.z, r.z);
        r.w = fmaf(w, v.w, r.w);
    }
    return r;
}

__global__ void fm_interp_kernel(FieldMapDev m, const float4 *pts, const int32_t *n_dev, int n, float4 *out,
                                 float3 e_ext)
{
    const int nn = n_dev ? *n_dev : n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    float4 r = fm_interp(m, pts[i]);
    r.x += e_ext.x;
    r.y += e_ext.y;
    r.z += e_ext.z;
    out[i] = r;
}

int obem_fieldmap_interp(obem_ctx *c, const float4 *pts, const int32_t *n_dev, int n, float4 *out, float3 e_ext,
                         cudaStream_t s)
{
    if (n <= 0) return OBEM_OK;
    fm_interp_kernel<<<(n + 255) / 256, 256, 0, s>>>(c->fm, pts, n_dev, n, out, e_ext);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}

int obem_fieldmap_build_nodes(obem_ctx *c, const float *sigma, cudaStream_t s)
{
    const size_t total = (size_t)c->fm.px * c->fm.py * c->fm.pz;
    float4 *pts = NULL;
    const int chunk = total < (size_t)FM_CHUNK ? (int)total : FM_CHUNK;
    OBEM_CUDA(c, cudaMalloc((void **)&pts, sizeof(float4) * (size_t)chunk));
    int rc = OBEM_OK;
    for (size_t first = 0; first < total && rc == OBEM_OK; first += chunk) {
        const int count = (int)(total - first < (size_t)chunk ? total - first : (size_t)chunk);
        fm_nodes_kernel<<<(count + 255) / 256, 256, 0, s>>>(c->fm, first, count, pts);
        FieldLaunch L;
        memset(&L, 0, sizeof L);
        L.targets = pts;
        L.nt = count;
        L.sigma = sigma;
        L.panels.c_a = c->d_c_a; L.panels.g0_h = c->d_g0_h; L.panels.g1 = c->d_g1; L.panels.g2 = c->d_g2;
        L.panels.nrm = c->d_nrm; L.panels.c_lo = c->d_c_lo; L.panels.v64 = c->d_v64; L.panels.geo = c->d_geo64;
        L.panels.np = c->np;
        L.E_out = c->fm.nodes + first;
        L.e_ext = make_float3(0.f, 0.f, 0.f);
        L.want_v = 1;
        rc = obem_launch_field(c, L, count, s);   // bricks in order: one cell-kernel block each
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(pts);
    if (rc != OBEM_OK) return rc;
    if (e != cudaSuccess) return obem_fail(c, OBEM_ERR_CUDA, "field map: %s", cudaGetErrorString(e));
    return OBEM_OK;
}
