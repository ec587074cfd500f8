// Host side of the far-cell groups (cellgroup.cu) run on the CPU: reads the
// cells (int np, double tri[np][9], float h2[np]) from argv[1], writes the
// group arrays to argv[2]: ng, perm[np], cr[ng][4], h2min[ng], u[M][4],
// c64[ng][4], v[C][3], pinv[M][C].  No CUDA call is made.
#include "../../paper_2110_09214_gb300/csrc/cellgroup.cu"

#include <stdio.h>

int obem_fail(obem_ctx *, int code, const char *, ...) { return code; }

static bool rd(void *p, size_t sz, size_t n, FILE *f) { return fread(p, sz, n, f) == n; }

int main(int argc, char **argv)
{
    if (argc < 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int np = 0;
    if (!rd(&np, 4, 1, f) || np <= 0) return 2;
    std::vector<double> tri(9 * (size_t)np);
    std::vector<float> h2(np);
    if (!rd(tri.data(), 8, tri.size(), f) || !rd(h2.data(), 4, h2.size(), f)) return 2;
    fclose(f);
    std::vector<float4> g0(np);
    for (int i = 0; i < np; ++i) g0[i] = make_float4(0.f, 0.f, 0.f, h2[i]);
    GroupHost H;
    const int rc = grp_host_build(tri.data(), g0.data(), np, H);
    if (rc != OBEM_OK) return 3;
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(&H.ng, 4, 1, o);
    fwrite(H.perm.data(), 4, np, o);
    fwrite(H.cr.data(), 16, H.ng, o);
    fwrite(H.h2min.data(), 4, H.ng, o);
    fwrite(H.u.data(), 16, OBEM_GRP_M, o);
    fwrite(H.c64.data(), 8, 4 * (size_t)H.ng, o);
    fwrite(H.vd.data(), 8, 3 * (size_t)OBEM_GRP_CHECK, o);
    fwrite(H.P.data(), 8, (size_t)OBEM_GRP_M * OBEM_GRP_CHECK, o);
    fclose(o);
    return 0;
}
