// Host side of the C ABI: context, gas and mesh loading, argument checks and
// dispatch to the kernels of field.cu, step.cu, bem.cu, backward.cu,
// fieldmap.cu, nn.cu and peak.cu (the batch of chambers is in batch.cu).
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>

#include "obem_internal.cuh"

int obem_fail(obem_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

static void free_dev(void *p)
{
    if (p) cudaFree(p);
}

static void free_mesh(obem_ctx *c)
{
    free(c->h_kind); free(c->h_group); free(c->h_tri); free(c->h_em); free(c->h_ep);
    c->h_kind = c->h_group = NULL;
    c->h_tri = c->h_em = c->h_ep = NULL;
    free_dev(c->d_c_a); free_dev(c->d_g0_h); free_dev(c->d_g1); free_dev(c->d_g2);
    free_dev(c->d_nrm); free_dev(c->d_c_lo); free_dev(c->d_v64); free_dev(c->d_kind); free_dev(c->d_group);
    free_dev(c->d_geo64);
    obem_cell_groups_free(c);
    obem_tc_free(c);
    free_dev(c->d_A); free_dev(c->d_LU); free_dev(c->d_piv); free_dev(c->d_rowscale);
    free_dev(c->d_work64); free_dev(c->d_work32); free_dev(c->d_flag); free_dev(c->d_sigma);
    free_dev(c->d_panel); free_dev(c->d_perm); free_dev(c->d_infl); free_dev(c->d_epsd); free_dev(c->d_trsv); free_dev(c->d_dinv);
    c->d_trsv = NULL;
    c->d_dinv = NULL;
    c->d_infl = c->d_epsd = NULL;
    c->d_panel = NULL;
    c->d_perm = NULL;
    free_dev(c->d_tri9); free_dev(c->d_hstart); free_dev(c->d_htri); free_dev(c->d_area); free_dev(c->d_deposit);
    c->d_tri9 = NULL;
    c->d_hstart = c->d_htri = NULL;
    c->d_area = NULL;
    c->d_deposit = NULL;
    c->d_c_a = c->d_g0_h = c->d_g1 = c->d_g2 = c->d_nrm = c->d_c_lo = NULL;
    c->d_v64 = NULL;
    c->d_kind = c->d_group = NULL;
    c->d_A = c->d_LU = NULL;
    c->d_piv = NULL;
    c->d_rowscale = NULL;
    c->d_work64 = NULL;
    c->d_work32 = NULL;
    c->d_flag = NULL;
    c->d_sigma = NULL;
    c->np = 0;
    c->factored = 0;
    c->nsys = c->nsys_alloc = 0;
    c->sigma_valid = 0;
}

extern "C" const char *obem_last_error(const obem_ctx *ctx)
{
    return ctx ? ctx->err : "null context";
}

extern "C" int obem_create(obem_ctx **out, const obem_config *cfg)
{
    if (!out || !cfg) return OBEM_ERR_ARG;
    *out = NULL;
    if (cfg->capacity < 1 || cfg->capacity > (1 << 30)) return OBEM_ERR_ARG;
    if (cfg->trial_cap < 1 || cfg->trial_cap > OBEM_MAX_TRIALS) return OBEM_ERR_ARG;
    if (cfg->nn_grid < 0 || cfg->nn_grid > OBEM_NN_GMAX) return OBEM_ERR_ARG;
    if (!(cfg->dt > 0.0) || !(cfg->softening >= 0.0) || !(cfg->z_lo < cfg->z_hi)) return OBEM_ERR_ARG;
    obem_ctx *c = (obem_ctx *)calloc(1, sizeof(obem_ctx));
    if (!c) return OBEM_ERR_ARG;
    c->cfg = *cfg;
    strcpy(c->err, "no error");
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        free(c);
        return OBEM_ERR_CUDA;
    }
    int cap = cfg->capacity;
    c->cap = cap;
    int max_blocks = (cap + 255) / 256 + 1;
    size_t bytes = 0;
#define ALLOC(p, n)                                                                     \
    do {                                                                                \
        if (cudaMalloc((void **)&(p), (size_t)(n)) != cudaSuccess) {                    \
            obem_destroy(c);                                                            \
            return OBEM_ERR_CUDA;                                                       \
        }                                                                               \
        bytes += (size_t)(n);                                                           \
    } while (0)
    ALLOC(c->s_E, sizeof(float4) * cap);
    ALLOC(c->s_prop, sizeof(unsigned long long) * cap);
    ALLOC(c->s_ionkey, sizeof(unsigned long long) * cap);
    ALLOC(c->s_keep, sizeof(int32_t) * cap);
    ALLOC(c->s_nsp, sizeof(int32_t) * cap);
    ALLOC(c->s_blk, sizeof(int32_t) * 4 * max_blocks);
    ALLOC(c->s_mpart, sizeof(double) * 13 * max_blocks);
    ALLOC(c->s_ctl, sizeof(StepCtl));
    ALLOC(c->o_pos, sizeof(float4) * cap);
    ALLOC(c->o_vel, sizeof(float4) * cap);
    ALLOC(c->o_id, sizeof(uint32_t) * cap);
    ALLOC(c->o_birth, sizeof(uint32_t) * cap);
    ALLOC(c->o_sp, cap);
    ALLOC(c->s_code, sizeof(uint32_t) * cap);
    ALLOC(c->s_perm, sizeof(int32_t) * cap);
    ALLOC(c->s_tk, sizeof(uint32_t) * cap);
    ALLOC(c->s_tv, sizeof(int32_t) * cap);
    ALLOC(c->s_rh, sizeof(int32_t) * (64 * (size_t)obem_binsort_blocks(cap) + 1));
    ALLOC(c->s_hist, sizeof(int32_t) * OBEM_NBINS);
    ALLOC(c->s_blocks, sizeof(int2) * ((size_t)cap / 512 + 2 + (cap < OBEM_NSUPER ? cap : OBEM_NSUPER)));
    ALLOC(c->s_nblocks, sizeof(int32_t) * (OBEM_NSUPER + 8));
    ALLOC(c->ph_count, sizeof(int32_t) * ((size_t)1 << 20));
    ALLOC(c->ph_start, sizeof(int32_t) * (((size_t)1 << 20) + 1));
    ALLOC(c->ph_cursor, sizeof(int32_t) * ((size_t)1 << 20));
    ALLOC(c->ph_bucket, sizeof(int32_t) * cap);
    ALLOC(c->ph_sorted, sizeof(int32_t) * cap);
    ALLOC(c->ph_bsum, sizeof(int32_t) * (1024 + 1));
    ALLOC(c->nn_bbox, sizeof(int) * 8);
    ALLOC(c->s_hit, sizeof(int32_t) * cap);
    ALLOC(c->nn_cell, sizeof(int32_t) * cap);
    ALLOC(c->nn_sorted, sizeof(int32_t) * cap);
    ALLOC(c->nn_count, sizeof(int32_t) * (size_t)OBEM_NN_GMAX * OBEM_NN_GMAX * OBEM_NN_GMAX);
    ALLOC(c->nn_start, sizeof(int32_t) * ((size_t)OBEM_NN_GMAX * OBEM_NN_GMAX * OBEM_NN_GMAX + 1));
    ALLOC(c->nn_cursor, sizeof(int32_t) * (size_t)OBEM_NN_GMAX * OBEM_NN_GMAX * OBEM_NN_GMAX);
    ALLOC(c->nn_agg, sizeof(float4) * 2 * (size_t)OBEM_NN_GMAX * OBEM_NN_GMAX * OBEM_NN_GMAX);
#undef ALLOC
    // partial sums of the symmetric all-pairs kernel for one pass of
    // diagonals (they grow as capacity x 512 tiles) and the per-charge
    // accumulator of the passes, kept within a quarter of the free memory
    // (and 64 GB); with them the charge-sorted copy of the charges and its
    // permutation
    {
        const size_t jb = sizeof(float) * obem_sym_pass_jpart_floats(cap) + sizeof(double) * 4 * (size_t)cap,
                     ib = sizeof(float) * obem_sym_pass_ipart_floats(cap);
        const size_t nb = (size_t)obem_sym_part_blocks(cap) + 1, ntile = (size_t)obem_sym_tiles(cap);
        size_t fr = 0, tot = 0;
        c->sym_grid = obem_sym_grid(c->device);
        if (c->sym_grid > 0 && cudaMemGetInfo(&fr, &tot) == cudaSuccess && jb + ib <= fr / 4 &&
            jb + ib <= ((size_t)64 << 30)) {
            if (cudaMalloc((void **)&c->sym_jpart, jb - sizeof(double) * 4 * (size_t)cap) != cudaSuccess ||
                cudaMalloc((void **)&c->sym_acc, sizeof(double) * 4 * (size_t)cap) != cudaSuccess ||
                cudaMalloc((void **)&c->sym_ipart, ib) != cudaSuccess ||
                cudaMalloc((void **)&c->sym_counter, sizeof(int)) != cudaSuccess ||
                cudaMalloc((void **)&c->sym_sorted, sizeof(float4) * cap) != cudaSuccess ||
                cudaMalloc((void **)&c->sym_perm, sizeof(int32_t) * cap) != cudaSuccess ||
                cudaMalloc((void **)&c->sym_bcnt, sizeof(int32_t) * nb) != cudaSuccess ||
                cudaMalloc((void **)&c->sym_tileq, sizeof(float) * ntile) != cudaSuccess) {
                free_dev(c->sym_jpart); free_dev(c->sym_ipart); free_dev(c->sym_counter); free_dev(c->sym_acc);
                free_dev(c->sym_sorted); free_dev(c->sym_perm); free_dev(c->sym_bcnt); free_dev(c->sym_tileq);
                c->sym_jpart = c->sym_ipart = NULL;
                c->sym_acc = NULL;
                c->sym_counter = c->sym_perm = c->sym_bcnt = NULL;
                c->sym_sorted = NULL;
                c->sym_tileq = NULL;
                cudaGetLastError();
            } else {
                c->sym_cap = cap;
            }
        }
    }
    (void)bytes;
    *out = c;
    return OBEM_OK;
}

extern "C" void obem_destroy(obem_ctx *c)
{
    if (!c) return;
    free_mesh(c);
    free_dev(c->d_egrid); free_dev(c->d_xs);
    free_dev(c->s_E); free_dev(c->s_prop); free_dev(c->s_ionkey); free_dev(c->s_keep);
    free_dev(c->s_nsp); free_dev(c->s_blk); free_dev(c->s_ctl); free_dev(c->o_pos); free_dev(c->s_mpart);
    free_dev(c->o_vel); free_dev(c->o_id); free_dev(c->o_birth); free_dev(c->o_sp);
    free_dev(c->s_code); free_dev(c->s_perm); free_dev(c->s_hist); free_dev(c->s_blocks); free_dev(c->s_nblocks);
    free_dev(c->s_tk); free_dev(c->s_tv); free_dev(c->s_rh);
    free_dev(c->d_ib);
    free_dev(c->sym_jpart); free_dev(c->sym_ipart); free_dev(c->sym_counter); free_dev(c->sym_acc);
    free_dev(c->sym_sorted); free_dev(c->sym_perm); free_dev(c->sym_bcnt); free_dev(c->sym_tileq);
    free_dev(c->ph_count); free_dev(c->ph_start); free_dev(c->ph_cursor); free_dev(c->ph_bucket); free_dev(c->ph_sorted); free_dev(c->ph_bsum);
    free_dev(c->fm.nodes);
    free_dev(c->s_hit);
    free_dev(c->nn_bbox); free_dev(c->nn_cell); free_dev(c->nn_sorted); free_dev(c->nn_count);
    free_dev(c->nn_start); free_dev(c->nn_cursor); free_dev(c->nn_agg);
    if (c->cublas) cublasDestroy(c->cublas);
    if (c->prof_ev) {
        for (int i = 0; i < OBEM_PROF_EV * OBEM_PROF_MAX; ++i) cudaEventDestroy(c->prof_ev[i]);
        free(c->prof_ev);
    }
    free_dev(c->d_counters);
    free(c);
}

extern "C" int obem_profile(obem_ctx *c, int32_t enable)
{
    if (!c) return OBEM_ERR_ARG;
    if (enable && !c->prof_ev) {
        c->prof_ev = (cudaEvent_t *)calloc(OBEM_PROF_EV * OBEM_PROF_MAX, sizeof(cudaEvent_t));
        for (int i = 0; i < OBEM_PROF_EV * OBEM_PROF_MAX; ++i) OBEM_CUDA(c, cudaEventCreate(&c->prof_ev[i]));
        OBEM_CUDA(c, cudaMalloc((void **)&c->d_counters, sizeof(unsigned long long) * OBEM_NCOUNTERS));
    }
    if (enable) {
        OBEM_CUDA(c, cudaMemset(c->d_counters, 0, sizeof(unsigned long long) * OBEM_NCOUNTERS));
        c->prof_n = 0;
        c->launches = 0;
        c->steps_recorded = 0;
    }
    c->prof_on = enable == OBEM_PROFILE_TIMES ? OBEM_PROFILE_TIMES : (enable ? 1 : 0);
    return OBEM_OK;
}

extern "C" int obem_stage_times(obem_ctx *c, double *ms, int64_t *counts)
{
    if (!c || !ms || !counts) return OBEM_ERR_ARG;
    for (int k = 0; k < 5; ++k) ms[k] = 0.0;
    for (int k = 0; k < 2 + OBEM_NCOUNTERS; ++k) counts[k] = 0;
    if (!c->prof_ev) return OBEM_OK;
    int n = c->prof_n < OBEM_PROF_MAX ? c->prof_n : OBEM_PROF_MAX;
    for (int r = 0; r < n; ++r) {
        cudaEvent_t *e = c->prof_ev + OBEM_PROF_EV * r;
        OBEM_CUDA(c, cudaEventSynchronize(e[3]));
        float t;
        OBEM_CUDA(c, cudaEventElapsedTime(&t, e[0], e[1])); ms[0] += t;
        OBEM_CUDA(c, cudaEventElapsedTime(&t, e[1], e[2])); ms[1] += t;
        OBEM_CUDA(c, cudaEventElapsedTime(&t, e[2], e[3])); ms[2] += t;
        OBEM_CUDA(c, cudaEventElapsedTime(&t, e[0], e[3])); ms[3] += t;
        OBEM_CUDA(c, cudaEventElapsedTime(&t, e[4], e[5])); ms[4] += t;
    }
    unsigned long long h[OBEM_NCOUNTERS];
    OBEM_CUDA(c, cudaMemcpy(h, c->d_counters, sizeof h, cudaMemcpyDeviceToHost));
    counts[0] = n;
    counts[1] = c->launches;
    for (int k = 0; k < OBEM_NCOUNTERS; ++k) counts[2 + k] = (int64_t)h[k];
    OBEM_CUDA(c, cudaMemset(c->d_counters, 0, sizeof h));
    c->prof_n = 0;
    c->launches = 0;
    return OBEM_OK;
}

// Constants of the collision model, each computed in FP64 and rounded once.
static void derive_gas(obem_ctx *c)
{
    GasDev &g = c->gas;
    const obem_config &cf = c->cfg;
    double M = c->gas_M_amu > 0 ? c->gas_M_amu * OBEM_AMU : INFINITY;
    int Minf = isinf(M);
    g.dt = (float)cf.dt;
    g.nu_ion = (float)c->gas_nu_ion;
    g.half_nu_ion = (float)(0.5 * c->gas_nu_ion);
    g.E_therm = (float)(1.5 * OBEM_KB * c->gas_T / OBEM_QE);
    g.v_th_ion = Minf ? 0.0f : (float)sqrt(3.0 * OBEM_KB * c->gas_T / M);
    g.qm[OBEM_ELECTRON] = (float)(-OBEM_QE / OBEM_ME);
    g.qm[OBEM_CATION] = Minf ? 0.0f : (float)(OBEM_QE / M);
    g.qm[OBEM_ANION] = Minf ? 0.0f : (float)(-OBEM_QE / M);
    g.K_e = (float)(0.5 * OBEM_ME / OBEM_QE);
    g.two_m_over_M = Minf ? 0.0f : (float)(2.0 * OBEM_ME / M);
    g.KCE = (float)(OBEM_KC * OBEM_QE);
    g.N = (float)c->gas_N;
    g.z_lo = (float)cf.z_lo;
    g.z_hi = (float)cf.z_hi;
    g.seed_lo = (uint32_t)(cf.seed & 0xFFFFFFFFu);
    g.seed_hi = (uint32_t)(cf.seed >> 32);
    g.trial_cap = cf.trial_cap;
    g.coll_mode = (cf.flags & OBEM_STEP_PROB_COLLISION) ? 1 : 0;
    g.recomb_on = cf.beta >= 0.0;
    double rc = 0.0;
    if (cf.beta > 0.0) rc = cbrt(3.0 * cf.beta * cf.dt / (4.0 * OBEM_PI));
    else if (cf.beta == 0.0 && c->gas_thr_ioni > 0.0f) rc = OBEM_KC * OBEM_QE / (2.0 * (double)c->gas_thr_ioni);
    else if (cf.beta == 0.0) g.recomb_on = 0;
    g.rc2 = (float)(rc * rc);
}

extern "C" int obem_gas_load(obem_ctx *c, const obem_gas *gs)
{
    if (!c || !gs) return OBEM_ERR_ARG;
    if (gs->n_proc < 1 || gs->n_proc > OBEM_MAX_PROC || gs->n_energy < 2 || gs->n_energy > 4096)
        return obem_fail(c, OBEM_ERR_ARG, "gas: n_proc must be 1..%d, n_energy 2..4096", OBEM_MAX_PROC);
    if (!gs->energy_eV || !gs->sigma_m2 || !gs->kind || !gs->mode || !gs->threshold_eV || !gs->nu_const)
        return obem_fail(c, OBEM_ERR_ARG, "gas: null table pointer");
    for (int i = 0; i + 1 < gs->n_energy; ++i)
        if (!(gs->energy_eV[i] < gs->energy_eV[i + 1]))
            return obem_fail(c, OBEM_ERR_ARG, "gas: energy grid not increasing at %d", i);
    for (int j = 0; j < gs->n_proc; ++j) {
        if (gs->kind[j] < 0 || gs->kind[j] > 3 || gs->mode[j] < 0 || gs->mode[j] > 1)
            return obem_fail(c, OBEM_ERR_ARG, "gas: bad kind/mode of process %d", j);
    }
    if (!(gs->N >= 0.0) || !(gs->T >= 0.0) || !(gs->nu_ion >= 0.0))
        return obem_fail(c, OBEM_ERR_ARG, "gas: negative N, T or nu_ion");
    int ne = gs->n_energy, npr = gs->n_proc;
    free_dev(c->d_egrid); free_dev(c->d_xs);
    c->d_egrid = NULL; c->d_xs = NULL;
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_egrid, sizeof(float) * ne));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_xs, sizeof(float) * ne * npr));
    OBEM_CUDA(c, cudaMemcpy(c->d_egrid, gs->energy_eV, sizeof(float) * ne, cudaMemcpyHostToDevice));
    OBEM_CUDA(c, cudaMemcpy(c->d_xs, gs->sigma_m2, sizeof(float) * ne * npr, cudaMemcpyHostToDevice));
    GasDev &g = c->gas;
    memset(&g, 0, sizeof g);
    g.egrid = c->d_egrid;
    g.xs = c->d_xs;
    g.n_proc = npr;
    g.n_e = ne;
    c->gas_T = gs->T; c->gas_N = gs->N; c->gas_M_amu = gs->M_amu; c->gas_nu_ion = gs->nu_ion;
    c->gas_thr_ioni = 0.0f;
    for (int j = 0; j < npr; ++j) {
        g.kind[j] = gs->kind[j];
        g.mode[j] = gs->mode[j];
        g.thr[j] = gs->threshold_eV[j];
        g.nuc[j] = gs->nu_const[j];
        if (gs->kind[j] == OBEM_P_IONISATION && c->gas_thr_ioni == 0.0f) c->gas_thr_ioni = gs->threshold_eV[j];
    }
    // Majorant of the electron collision frequency for the null-collision
    // method: constant-frequency processes add their frequency; tabulated ones
    // are bounded on each grid segment by N max(sigma_tot) v(E_upper).
    double nuc = 0.0, best = 0.0;
    for (int j = 0; j < npr; ++j)
        if (gs->mode[j] == OBEM_MODE_CONST) nuc += (double)gs->nu_const[j];
    for (int i = 0; i + 1 < ne; ++i) {
        double s0 = 0.0, s1 = 0.0;
        for (int j = 0; j < npr; ++j) {
            if (gs->mode[j] != OBEM_MODE_TABLE) continue;
            s0 += (double)gs->sigma_m2[(size_t)j * ne + i];
            s1 += (double)gs->sigma_m2[(size_t)j * ne + i + 1];
        }
        double v1 = sqrt(2.0 * (double)gs->energy_eV[i + 1] * OBEM_QE / OBEM_ME);
        double b = gs->N * (s0 > s1 ? s0 : s1) * v1;
        if (b > best) best = b;
    }
    g.nu_max_e = (float)(nuc + best);
    derive_gas(c);
    c->gas_loaded = 1;
    return OBEM_OK;
}

// FP64 geometry of each cell for the closed form: unit normal n, twice the
// area |(v1 - v0) x (v2 - v0)|, and for each edge i -> i+1 its unit vector and
// its in-plane normal (edge x n); OBEM_GEO64 doubles per cell.
void obem_cell_geo64(const double *tri, int np, double *geo)
{
    for (int i = 0; i < np; ++i) {
        const double *v = tri + 9 * (size_t)i;
        double *g = geo + (size_t)OBEM_GEO64 * i;
        const double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        const double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double a2 = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int k = 0; k < 3; ++k) n[k] /= a2;
        g[0] = n[0]; g[1] = n[1]; g[2] = n[2]; g[3] = a2;
        for (int e = 0; e < 3; ++e) {
            const int j = (e + 1) % 3;
            double d[3] = {v[3 * j] - v[3 * e], v[3 * j + 1] - v[3 * e + 1], v[3 * j + 2] - v[3 * e + 2]};
            const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int k = 0; k < 3; ++k) d[k] /= len;
            double *gd = g + 4 + 6 * e;
            gd[0] = d[0]; gd[1] = d[1]; gd[2] = d[2];
            gd[3] = d[1] * n[2] - d[2] * n[1];
            gd[4] = d[2] * n[0] - d[0] * n[2];
            gd[5] = d[0] * n[1] - d[1] * n[0];
        }
        g[22] = 0.0; g[23] = 0.0;
    }
}

// Cell geometry in the layout of the field kernels (see PanelsDev) from FP64
// vertices; kind may be NULL (electrode).  Returns the first degenerate cell,
// or -1.
int obem_cell_layout(const double *tri, const int32_t *kind, int np, float4 *ca, float4 *g0, float4 *g1,
                     float4 *g2, float4 *nr, float4 *cl)
{
    for (int i = 0; i < np; ++i) {
        const double *v = tri + 9 * (size_t)i;
        double cc[3], e1[3], e2[3], nn[3];
        for (int k = 0; k < 3; ++k) {
            cc[k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0;
            e1[k] = v[3 + k] - v[k];
            e2[k] = v[6 + k] - v[k];
        }
        nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double a2 = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        if (!(a2 > 0.0)) return i;
        double h2 = 0.0;
        for (int e = 0; e < 3; ++e) {
            const double *a = v + 3 * e, *b = v + 3 * ((e + 1) % 3);
            double d = (a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]);
            if (d > h2) h2 = d;
        }
        ca[i] = make_float4((float)cc[0], (float)cc[1], (float)cc[2], (float)(OBEM_KC * 0.5 * a2));
        g0[i] = make_float4((float)(v[0] - cc[0]), (float)(v[1] - cc[1]), (float)(v[2] - cc[2]), (float)h2);
        g1[i] = make_float4((float)(v[3] - cc[0]), (float)(v[4] - cc[1]), (float)(v[5] - cc[2]), 0.f);
        g2[i] = make_float4((float)(v[6] - cc[0]), (float)(v[7] - cc[1]), (float)(v[8] - cc[2]), 0.f);
        nr[i] = make_float4((float)(nn[0] / a2), (float)(nn[1] / a2), (float)(nn[2] / a2),
                            (float)(kind ? kind[i] : OBEM_CELL_ELECTRODE));
        cl[i] = make_float4((float)(cc[0] - (double)ca[i].x), (float)(cc[1] - (double)ca[i].y),
                            (float)(cc[2] - (double)ca[i].z), 0.f);
    }
    return -1;
}

extern "C" int obem_mesh_load(obem_ctx *c, int32_t np, const double *tri, const int32_t *kind,
                              const int32_t *group, const double *em, const double *ep,
                              int32_t n_groups)
{
    if (!c) return OBEM_ERR_ARG;
    if (np < 1 || np > 200000) return obem_fail(c, OBEM_ERR_ARG, "mesh: n_panels must be 1..200000");
    if (!tri || !kind || !group || !em || !ep) return obem_fail(c, OBEM_ERR_ARG, "mesh: null array");
    if (n_groups < 0) return obem_fail(c, OBEM_ERR_ARG, "mesh: n_groups < 0");
    for (int i = 0; i < np; ++i) {
        if (kind[i] != OBEM_CELL_ELECTRODE && kind[i] != OBEM_CELL_DIELECTRIC)
            return obem_fail(c, OBEM_ERR_ARG, "mesh: bad kind of cell %d", i);
        if (kind[i] == OBEM_CELL_ELECTRODE && (group[i] < 0 || group[i] >= n_groups))
            return obem_fail(c, OBEM_ERR_ARG, "mesh: cell %d has group %d outside 0..%d", i, group[i], n_groups - 1);
    }
    free_mesh(c);
    c->np = np;
    c->n_groups = n_groups;
    c->h_kind = (int *)malloc(sizeof(int) * np);
    c->h_group = (int *)malloc(sizeof(int) * np);
    c->h_tri = (double *)malloc(sizeof(double) * 9 * np);
    c->h_em = (double *)malloc(sizeof(double) * np);
    c->h_ep = (double *)malloc(sizeof(double) * np);
    memcpy(c->h_kind, kind, sizeof(int) * np);
    memcpy(c->h_group, group, sizeof(int) * np);
    memcpy(c->h_tri, tri, sizeof(double) * 9 * np);
    memcpy(c->h_em, em, sizeof(double) * np);
    memcpy(c->h_ep, ep, sizeof(double) * np);
    for (int k = 0; k < 3; ++k) { c->bbox_lo[k] = 3e38f; c->bbox_hi[k] = -3e38f; }
    for (int i = 0; i < np; ++i)
        for (int v = 0; v < 3; ++v)
            for (int k = 0; k < 3; ++k) {
                float x = (float)tri[9 * (size_t)i + 3 * v + k];
                if (x < c->bbox_lo[k]) c->bbox_lo[k] = x;
                if (x > c->bbox_hi[k]) c->bbox_hi[k] = x;
            }
    float4 *ca = (float4 *)malloc(sizeof(float4) * np);
    float4 *g0 = (float4 *)malloc(sizeof(float4) * np);
    float4 *g1 = (float4 *)malloc(sizeof(float4) * np);
    float4 *g2 = (float4 *)malloc(sizeof(float4) * np);
    float4 *nr = (float4 *)malloc(sizeof(float4) * np);
    float4 *cl = (float4 *)malloc(sizeof(float4) * np);
    const int bad = obem_cell_layout(tri, kind, np, ca, g0, g1, g2, nr, cl);
    if (bad >= 0) {
        free(ca); free(g0); free(g1); free(g2); free(nr); free(cl);
        free_mesh(c);
        return obem_fail(c, OBEM_ERR_ARG, "mesh: cell %d is degenerate", bad);
    }
    int rc = OBEM_OK;
    size_t f4 = sizeof(float4) * np;
#define UP(dst, src, bytes)                                                              \
    do {                                                                                 \
        if (rc == OBEM_OK && (cudaMalloc((void **)&(dst), (bytes)) != cudaSuccess ||     \
                              cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice)  \
                                  != cudaSuccess))                                       \
            rc = obem_fail(c, OBEM_ERR_CUDA, "mesh upload failed");                      \
    } while (0)
    UP(c->d_c_a, ca, f4);
    UP(c->d_g0_h, g0, f4);
    UP(c->d_g1, g1, f4);
    UP(c->d_g2, g2, f4);
    UP(c->d_nrm, nr, f4);
    UP(c->d_c_lo, cl, f4);
    UP(c->d_v64, tri, sizeof(double) * 9 * np);
    {
        double *geo = (double *)malloc(sizeof(double) * OBEM_GEO64 * np);
        if (!geo) rc = obem_fail(c, OBEM_ERR_ARG, "mesh: host allocation failed");
        else {
            obem_cell_geo64(tri, np, geo);
            UP(c->d_geo64, geo, sizeof(double) * OBEM_GEO64 * np);
            free(geo);
        }
    }
    UP(c->d_kind, kind, sizeof(int) * np);
    UP(c->d_group, group, sizeof(int) * np);
    // charging-up: binary32 vertices, areas, and a uniform grid over the
    // cells (cubic grid cells of about two mean cell sizes, at most 256 per
    // axis; each cell listed in every grid cell its bounding box touches,
    // padded by one grid cell on every side)
    {
        float *t9 = (float *)malloc(sizeof(float) * 9 * np);
        double *ar = (double *)malloc(sizeof(double) * np);
        double mean_h = 0.0;
        for (int i = 0; i < np; ++i) {
            const double *v = tri + 9 * (size_t)i;
            for (int k = 0; k < 9; ++k) t9[9 * (size_t)i + k] = (float)v[k];
            double e1[3], e2[3];
            for (int k = 0; k < 3; ++k) { e1[k] = v[3 + k] - v[k]; e2[k] = v[6 + k] - v[k]; }
            const double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
                         nz = e1[0] * e2[1] - e1[1] * e2[0];
            ar[i] = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
            mean_h += sqrt(2.0 * ar[i]);
        }
        mean_h /= np;
        float ext = 0.0f;
        for (int k = 0; k < 3; ++k) {
            c->h_hlo[k] = c->bbox_lo[k];
            ext = fmaxf(ext, c->bbox_hi[k] - c->bbox_lo[k]);
        }
        float cellw = (float)(2.0 * mean_h);
        if (!(cellw > ext / 256.0f)) cellw = ext / 256.0f;
        if (!(cellw > 0.0f)) cellw = 1.0f;
        c->h_hinv = 1.0f / cellw;
        size_t ncell = 1;
        for (int k = 0; k < 3; ++k) {
            int d = (int)floorf((c->bbox_hi[k] - c->h_hlo[k]) * c->h_hinv) + 1;
            c->h_hdim[k] = d < 1 ? 1 : (d > 256 ? 256 : d);
            ncell *= (size_t)c->h_hdim[k];
        }
        auto coord = [&](float x, int k) {
            int q = (int)floorf((x - c->h_hlo[k]) * c->h_hinv);
            return q < 0 ? 0 : (q > c->h_hdim[k] - 1 ? c->h_hdim[k] - 1 : q);
        };
        int32_t *cnt = (int32_t *)calloc(ncell + 1, sizeof(int32_t));
        for (int pass = 0; pass < 2; ++pass) {
            int32_t *lst = NULL;
            if (pass == 1) {
                for (size_t q = 0, run = 0; q <= ncell; ++q) { int32_t t = cnt[q]; cnt[q] = (int32_t)run; run += t; }
                lst = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cnt[ncell] + 1));
            }
            int32_t *cur = pass == 1 ? (int32_t *)malloc(sizeof(int32_t) * (ncell + 1)) : NULL;
            if (cur) memcpy(cur, cnt, sizeof(int32_t) * (ncell + 1));
            for (int i = 0; i < np; ++i) {
                int lo3[3], hi3[3];
                for (int k = 0; k < 3; ++k) {
                    float mn = t9[9 * (size_t)i + k], mx = mn;
                    for (int v = 1; v < 3; ++v) {
                        mn = fminf(mn, t9[9 * (size_t)i + 3 * v + k]);
                        mx = fmaxf(mx, t9[9 * (size_t)i + 3 * v + k]);
                    }
                    lo3[k] = coord(mn, k) - 1; hi3[k] = coord(mx, k) + 1;
                    if (lo3[k] < 0) lo3[k] = 0;
                    if (hi3[k] > c->h_hdim[k] - 1) hi3[k] = c->h_hdim[k] - 1;
                }
                for (int z = lo3[2]; z <= hi3[2]; ++z)
                    for (int y = lo3[1]; y <= hi3[1]; ++y)
                        for (int x = lo3[0]; x <= hi3[0]; ++x) {
                            size_t q = ((size_t)z * c->h_hdim[1] + y) * c->h_hdim[0] + x;
                            if (pass == 0) cnt[q] += 1;
                            else lst[cur[q]++] = i;
                        }
            }
            if (pass == 1) {
                UP(c->d_htri, lst, sizeof(int32_t) * ((size_t)cnt[ncell] + 1));
                UP(c->d_hstart, cnt, sizeof(int32_t) * (ncell + 1));
                free(lst);
                free(cur);
            }
        }
        UP(c->d_tri9, t9, sizeof(float) * 9 * np);
        UP(c->d_area, ar, sizeof(double) * np);
        free(cnt); free(t9); free(ar);
        if (rc == OBEM_OK && (cudaMalloc((void **)&c->d_deposit, sizeof(long long) * np) != cudaSuccess ||
                              cudaMemset(c->d_deposit, 0, sizeof(long long) * np) != cudaSuccess))
            rc = obem_fail(c, OBEM_ERR_CUDA, "mesh: deposit allocation failed");
    }
#undef UP
    if (rc == OBEM_OK && (c->cfg.flags & OBEM_STEP_CELL_GROUPS))
        rc = obem_cell_groups_build(c, tri, g0, np);
    free(ca); free(g0); free(g1); free(g2); free(nr); free(cl);
    if (rc == OBEM_OK && cudaMalloc((void **)&c->d_sigma, sizeof(float) * np) != cudaSuccess)
        rc = obem_fail(c, OBEM_ERR_CUDA, "mesh: sigma allocation failed");
    if (rc != OBEM_OK) free_mesh(c);
    return rc;
}

static PanelsDev panels_of(const obem_ctx *c)
{
    PanelsDev p;
    p.c_a = c->d_c_a; p.g0_h = c->d_g0_h; p.g1 = c->d_g1; p.g2 = c->d_g2; p.nrm = c->d_nrm;
    p.c_lo = c->d_c_lo;
    p.v64 = c->d_v64;
    p.geo = c->d_geo64;
    p.np = c->np;
    return p;
}

extern "C" int obem_bem_assemble(obem_ctx *c, int32_t precision, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (c->np < 1) return obem_fail(c, OBEM_ERR_STATE, "assemble: no mesh loaded");
    if (precision < OBEM_LU_FP32 || precision > OBEM_LU_BF16X9)
        return obem_fail(c, OBEM_ERR_ARG, "assemble: unknown precision %d", precision);
    return obem_assemble_and_factor(c, precision, (cudaStream_t)stream);
}

extern "C" int obem_bem_solve(obem_ctx *c, const double *gv, const float *sigma_free,
                              const float *drhs, float *sigma_out, obem_solve_report *rep,
                              obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (!c->factored) return obem_fail(c, OBEM_ERR_STATE, "solve: call obem_bem_assemble first");
    if (c->n_groups > 0 && !gv) return obem_fail(c, OBEM_ERR_ARG, "solve: group_voltage is NULL");
    if (!sigma_out) return obem_fail(c, OBEM_ERR_ARG, "solve: sigma_out is NULL");
    return obem_solve_system(c, gv, sigma_free, drhs, sigma_out, rep, (cudaStream_t)stream);
}

extern "C" int obem_dense_factor(obem_ctx *c, const float *A, int32_t n, int32_t precision, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (c->np > 0) return obem_fail(c, OBEM_ERR_STATE, "dense factor: the context holds a mesh");
    if (!A || n < 1) return obem_fail(c, OBEM_ERR_ARG, "dense factor: no matrix");
    if (precision < OBEM_LU_FP32 || precision > OBEM_LU_BF16X9)
        return obem_fail(c, OBEM_ERR_ARG, "dense factor: unknown precision %d", precision);
    return obem_factor_dense(c, A, n, precision, (cudaStream_t)stream);
}

extern "C" int obem_dense_solve(obem_ctx *c, const double *b, double *x, obem_solve_report *rep,
                                obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (c->np > 0 || !c->factored) return obem_fail(c, OBEM_ERR_STATE, "dense solve: call obem_dense_factor first");
    if (!b || !x) return obem_fail(c, OBEM_ERR_ARG, "dense solve: null b or x");
    return obem_solve_dense_rhs(c, b, x, rep, (cudaStream_t)stream);
}

extern "C" int obem_bem_solve_adjoint(obem_ctx *c, const float *dL_dsigma, double *dL_dgroup_voltage,
                                      float *dL_db, obem_solve_report *rep, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (!c->factored) return obem_fail(c, OBEM_ERR_STATE, "solve adjoint: call obem_bem_assemble first");
    if (!dL_dsigma) return obem_fail(c, OBEM_ERR_ARG, "solve adjoint: dL_dsigma is NULL");
    return obem_solve_adjoint(c, dL_dsigma, dL_dgroup_voltage, dL_db, rep, (cudaStream_t)stream);
}

extern "C" int obem_field_eval(obem_ctx *c, const float *targets, int32_t nt, const float *sources,
                               int32_t ns, int32_t self_exclude, const float *sigma, float *E_out,
                               obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (nt < 0 || (sources && ns < 0)) return obem_fail(c, OBEM_ERR_ARG, "field: negative count");
    if (nt == 0) return OBEM_OK;
    if (!targets || !E_out) return obem_fail(c, OBEM_ERR_ARG, "field: null targets or E_out");
    if (self_exclude && (!sources || ns != nt))
        return obem_fail(c, OBEM_ERR_ARG, "field: self_exclude needs sources with ns == nt");
    if (sigma && c->np < 1) return obem_fail(c, OBEM_ERR_STATE, "field: sigma given but no mesh loaded");
    if (((uintptr_t)targets | (uintptr_t)E_out | (uintptr_t)sources) & 15)
        return obem_fail(c, OBEM_ERR_ARG, "field: arrays must be 16-byte aligned");
    FieldLaunch L;
    memset(&L, 0, sizeof L);
    L.targets = (const float4 *)targets;
    L.nt = nt;
    L.sources = (sources && ns > 0) ? (const float4 *)sources : NULL;
    L.ns = ns;
    L.self_exclude = self_exclude ? 1 : 0;
    L.eps2 = 0.0f;
    L.sigma = sigma;
    L.panels = panels_of(c);
    L.E_out = (float4 *)E_out;
    L.e_ext = make_float3(0.f, 0.f, 0.f);
    L.want_v = 1;
    // the scratch holds a spatial order for up to `capacity` targets; larger
    // calls keep the given order (same results, slower cell kernel)
    L.perm = (sigma && nt <= c->cap) ? c->s_perm : NULL;
    L.blocks = L.perm ? c->s_blocks : NULL;
    L.nblocks = L.perm ? c->s_nblocks : NULL;
    return obem_launch_field(c, L, nt, (cudaStream_t)stream);
}

extern "C" int obem_field_eval_backward(obem_ctx *c, const float *targets, int32_t nt, const float *sources,
                                        int32_t ns, int32_t self_exclude, const float *sigma,
                                        const float *dL_dE, float *dL_dsigma, float *dL_dtargets,
                                        float *dL_dsources, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (nt < 0 || (sources && ns < 0)) return obem_fail(c, OBEM_ERR_ARG, "field backward: negative count");
    if (self_exclude && (!sources || ns != nt))
        return obem_fail(c, OBEM_ERR_ARG, "field backward: self_exclude needs sources with ns == nt");
    if (dL_dsources && !sources)
        return obem_fail(c, OBEM_ERR_ARG, "field backward: dL_dsources needs sources");
    if ((sigma || dL_dsigma) && c->np < 1)
        return obem_fail(c, OBEM_ERR_STATE, "field backward: sigma or dL_dsigma given but no mesh loaded");
    if (nt > 0 && (!targets || !dL_dE))
        return obem_fail(c, OBEM_ERR_ARG, "field backward: null targets or dL_dE");
    if (((uintptr_t)targets | (uintptr_t)sources | (uintptr_t)dL_dE | (uintptr_t)dL_dtargets |
         (uintptr_t)dL_dsources) & 15)
        return obem_fail(c, OBEM_ERR_ARG, "field backward: arrays must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (nt == 0) {
        // sums over no targets
        if (dL_dsigma) OBEM_CUDA(c, cudaMemsetAsync(dL_dsigma, 0, sizeof(float) * (size_t)c->np, s));
        if (dL_dsources && ns > 0) OBEM_CUDA(c, cudaMemsetAsync(dL_dsources, 0, sizeof(float) * 4 * (size_t)ns, s));
        return OBEM_OK;
    }
    BwArgs A;
    memset(&A, 0, sizeof A);
    A.targets = targets;
    A.nt = nt;
    A.sources = (sources && ns > 0) ? sources : NULL;
    A.ns = A.sources ? ns : 0;
    A.self_exclude = self_exclude ? 1 : 0;
    A.sigma = sigma;
    A.panels = panels_of(c);
    A.dL_dE = dL_dE;
    A.dL_dsigma = dL_dsigma;
    A.dL_dtargets = dL_dtargets;
    A.dL_dsources = dL_dsources;
    return obem_launch_backward(c, A, s);
}

// ---------------------------------------------------------------- sharded step
static int shard_state_ok(obem_ctx *c, const obem_state *st, const char *who)
{
    if (!st) return obem_fail(c, OBEM_ERR_ARG, "%s: null state", who);
    if (!st->pos_q || !st->vel || !st->id || !st->birth || !st->species || !st->n || !st->next_id)
        return obem_fail(c, OBEM_ERR_ARG, "%s: null state array", who);
    if (st->capacity < 1 || st->capacity > c->cap)
        return obem_fail(c, OBEM_ERR_ARG, "%s: state capacity %d outside 1..%d", who, st->capacity, c->cap);
    if (((uintptr_t)st->pos_q | (uintptr_t)st->vel) & 15)
        return obem_fail(c, OBEM_ERR_ARG, "%s: pos_q / vel must be 16-byte aligned", who);
    return OBEM_OK;
}

extern "C" int obem_shard_field(obem_ctx *c, const obem_state *st, const float *sources, int32_t ns, int32_t self_off,
                                float *E_out, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    int rc = shard_state_ok(c, st, "shard field");
    if (rc != OBEM_OK) return rc;
    if (!E_out || ns < 0 || (ns > 0 && !sources) || self_off < 0 || self_off > ns)
        return obem_fail(c, OBEM_ERR_ARG, "shard field: bad sources, offset or output");
    if (((uintptr_t)sources | (uintptr_t)E_out) & 15)
        return obem_fail(c, OBEM_ERR_ARG, "shard field: sources / E_out must be 16-byte aligned");
    if (c->cfg.flags & (OBEM_STEP_FIELD_MAP | OBEM_STEP_NBODY_NN))
        return obem_fail(c, OBEM_ERR_ARG, "shard field: the static map and the approximate N-body field are not sharded");
    const int want_cells = (c->cfg.flags & OBEM_STEP_CELL_FIELD) && c->sigma_valid;
    const int want_nbody = (c->cfg.flags & OBEM_STEP_SPACE_CHARGE) && ns > 0;
    FieldLaunch L;
    memset(&L, 0, sizeof L);
    L.targets = (const float4 *)st->pos_q;
    L.nt_dev = st->n;
    L.nt = st->capacity;
    L.sources = want_nbody ? (const float4 *)sources : NULL;
    L.ns = ns;
    L.self_exclude = 1;
    L.self_off = self_off;
    L.shard = 1;
    L.eps2 = (float)(c->cfg.softening * c->cfg.softening);
    L.sigma = want_cells ? c->d_sigma : NULL;
    L.panels = panels_of(c);
    L.perm = want_cells ? c->s_perm : NULL;
    L.blocks = want_cells ? c->s_blocks : NULL;
    L.nblocks = want_cells ? c->s_nblocks : NULL;
    L.E_out = (float4 *)E_out;
    L.e_ext = make_float3((float)c->cfg.e_ext[0], (float)c->cfg.e_ext[1], (float)c->cfg.e_ext[2]);
    return obem_launch_field(c, L, st->capacity, (cudaStream_t)stream);
}

extern "C" int obem_shard_propose(obem_ctx *c, const obem_state *st, const obem_state *gathered, uint32_t step,
                                  int64_t *ionkey, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (!c->gas_loaded) return obem_fail(c, OBEM_ERR_STATE, "shard propose: call obem_gas_load first");
    int rc = shard_state_ok(c, st, "shard propose");
    if (rc == OBEM_OK) rc = shard_state_ok(c, gathered, "shard propose (gathered)");
    if (rc != OBEM_OK) return rc;
    if (!ionkey) return obem_fail(c, OBEM_ERR_ARG, "shard propose: null ionkey");
    return obem_launch_shard_propose(c, st, gathered, step, (unsigned long long *)ionkey, (cudaStream_t)stream);
}

extern "C" int obem_shard_count(obem_ctx *c, const obem_state *st, const float *E, uint32_t step,
                                const int64_t *ionkey, int32_t self_off, obem_step_stats *stats, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (!c->gas_loaded) return obem_fail(c, OBEM_ERR_STATE, "shard count: call obem_gas_load first");
    int rc = shard_state_ok(c, st, "shard count");
    if (rc != OBEM_OK) return rc;
    if (!E || !ionkey || !stats || self_off < 0 || ((uintptr_t)E & 15))
        return obem_fail(c, OBEM_ERR_ARG, "shard count: bad field, keys, stats or offset");
    return obem_launch_shard_count(c, st, (const float4 *)E, step, (const unsigned long long *)ionkey, self_off, stats,
                                   (cudaStream_t)stream);
}

extern "C" int obem_shard_commit(obem_ctx *c, const obem_state *st, const float *E, uint32_t step, uint32_t id_base,
                                 int32_t commit, obem_step_stats *stats, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    int rc = shard_state_ok(c, st, "shard commit");
    if (rc != OBEM_OK) return rc;
    if (!E || !stats || ((uintptr_t)E & 15)) return obem_fail(c, OBEM_ERR_ARG, "shard commit: bad field or stats");
    return obem_launch_shard_commit(c, st, (const float4 *)E, step, id_base, commit ? 1 : 0, stats,
                                    (cudaStream_t)stream);
}

static int influence(obem_ctx *c, const float *sources, int32_t ns, float *drhs, int selftest, cudaStream_t s)
{
    if (!c->d_infl) {
        // first call: the per-cell sums and eps+ - eps- of the dielectric cells
        OBEM_CUDA(c, cudaMalloc((void **)&c->d_infl, sizeof(double) * 4 * (size_t)c->np));
        OBEM_CUDA(c, cudaMalloc((void **)&c->d_epsd, sizeof(double) * (size_t)c->np));
        double *h = (double *)malloc(sizeof(double) * (size_t)c->np);
        if (!h) return obem_fail(c, OBEM_ERR_ARG, "influence: host allocation failed");
        for (int i = 0; i < c->np; ++i)
            h[i] = c->h_kind[i] == OBEM_CELL_DIELECTRIC ? c->h_ep[i] - c->h_em[i] : 0.0;
        cudaError_t e = cudaMemcpy(c->d_epsd, h, sizeof(double) * (size_t)c->np, cudaMemcpyHostToDevice);
        free(h);
        OBEM_CUDA(c, e);
    }
    const size_t need = obem_influence_scratch_bytes(ns, c->np);
    if (ns > 0 && need > c->ib_bytes) {
        free_dev(c->d_ib);
        c->d_ib = NULL;
        c->ib_bytes = 0;
        OBEM_CUDA(c, cudaMalloc(&c->d_ib, need));
        c->ib_bytes = need;
    }
    return obem_launch_influence(c, (const float4 *)sources, ns, panels_of(c), c->d_infl, c->d_geo64, c->d_kind,
                                 c->d_epsd, drhs, c->d_ib, selftest, s);
}

extern "C" int obem_influence_rhs(obem_ctx *c, const float *sources, int32_t ns, float *drhs, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (c->np < 1) return obem_fail(c, OBEM_ERR_STATE, "influence: no mesh loaded");
    if (ns < 0 || (ns > 0 && !sources) || !drhs) return obem_fail(c, OBEM_ERR_ARG, "influence: bad arguments");
    if ((uintptr_t)sources & 15) return obem_fail(c, OBEM_ERR_ARG, "influence: sources must be 16-byte aligned");
    return influence(c, sources, ns, drhs, 0, (cudaStream_t)stream);
}

extern "C" int obem_selftest_waits(obem_ctx *c, int32_t which, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (which == 0) return obem_selftest_wait_timeout(c, stream);
    if (which == 1) return obem_selftest_solve_wait(c, s);
    if (which != 2) return obem_fail(c, OBEM_ERR_ARG, "wait self-test: no wait %d", which);
    if (c->np < 1) return obem_fail(c, OBEM_ERR_STATE, "wait self-test: no mesh loaded");
    // the cells' centroids (weights as charges) as sources: the values do not
    // matter, every bulk copy's barrier expects 16 bytes more than it gets
    float *drhs = NULL;
    OBEM_CUDA(c, cudaMalloc((void **)&drhs, sizeof(float) * (size_t)c->np));
    const int rc = influence(c, (const float *)panels_of(c).c_a, c->np, drhs, 1, s);
    cudaFree(drhs);
    if (rc == OBEM_ERR_TIMEOUT) {
        c->err[0] = 0;
        return OBEM_OK;
    }
    if (rc != OBEM_OK) return rc;
    return obem_fail(c, OBEM_ERR_STATE, "wait self-test: the influence pass reported no timeout");
}

extern "C" int obem_surface_charge(obem_ctx *c, float *sigma_free, int64_t *counts, int32_t reset,
                                   obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (c->np < 1 || !c->d_deposit) return obem_fail(c, OBEM_ERR_STATE, "surface charge: no mesh loaded");
    cudaStream_t s = (cudaStream_t)stream;
    if (sigma_free) {
        int rc = obem_launch_surface_sigma(c, sigma_free, s);
        if (rc != OBEM_OK) return rc;
    }
    if (counts) {
        OBEM_CUDA(c, cudaMemcpyAsync(counts, c->d_deposit, sizeof(long long) * c->np, cudaMemcpyDeviceToHost, s));
        OBEM_CUDA(c, cudaStreamSynchronize(s));
    }
    if (reset) OBEM_CUDA(c, cudaMemsetAsync(c->d_deposit, 0, sizeof(long long) * c->np, s));
    return OBEM_OK;
}

extern "C" int obem_nbody_nn_eval(obem_ctx *c, const float *pos_q, int32_t n, int32_t grid, double softening,
                                  float *E_out, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (n < 0 || n > c->cap) return obem_fail(c, OBEM_ERR_ARG, "nbody NN: n %d outside 0..%d (capacity)", n, c->cap);
    if (grid < 1 || grid > OBEM_NN_GMAX)
        return obem_fail(c, OBEM_ERR_ARG, "nbody NN: grid %d outside 1..%d", grid, OBEM_NN_GMAX);
    if (!(softening >= 0.0)) return obem_fail(c, OBEM_ERR_ARG, "nbody NN: negative softening");
    if (n == 0) return OBEM_OK;
    if (!pos_q || !E_out) return obem_fail(c, OBEM_ERR_ARG, "nbody NN: null pos_q or E_out");
    if (((uintptr_t)pos_q | (uintptr_t)E_out) & 15)
        return obem_fail(c, OBEM_ERR_ARG, "nbody NN: arrays must be 16-byte aligned");
    return obem_launch_nbody_nn(c, (const float4 *)pos_q, NULL, n, grid, (float)(softening * softening),
                                (float4 *)E_out, make_float3(0.f, 0.f, 0.f), 0, (cudaStream_t)stream);
}

extern "C" int obem_fieldmap_build(obem_ctx *c, const double *lo, const double *hi, const int32_t *dims,
                                   const float *sigma, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (c->np < 1) return obem_fail(c, OBEM_ERR_STATE, "field map: no mesh loaded");
    if (!lo || !hi || !dims || !sigma) return obem_fail(c, OBEM_ERR_ARG, "field map: null argument");
    size_t total = 1;
    int pad[3];
    for (int a = 0; a < 3; ++a) {
        if (!(hi[a] > lo[a]) || dims[a] < 2 || dims[a] > (1 << 16))
            return obem_fail(c, OBEM_ERR_ARG, "field map: axis %d needs lo < hi and 2 <= dims <= 65536", a);
        pad[a] = (dims[a] + 7) / 8 * 8;
        total *= (size_t)pad[a];
    }
    if (total > ((size_t)1 << 31)) return obem_fail(c, OBEM_ERR_ARG, "field map: more than 2^31 nodes");
    free_dev(c->fm.nodes);
    memset(&c->fm, 0, sizeof c->fm);
    float4 *nodes = NULL;
    OBEM_CUDA(c, cudaMalloc((void **)&nodes, sizeof(float4) * total));
    c->fm.nodes = nodes;
    c->fm.nx = dims[0]; c->fm.ny = dims[1]; c->fm.nz = dims[2];
    c->fm.px = pad[0]; c->fm.py = pad[1]; c->fm.pz = pad[2];
    for (int a = 0; a < 3; ++a) {
        c->fm.lo[a] = lo[a];
        c->fm.step[a] = (hi[a] - lo[a]) / (double)(dims[a] - 1);
    }
    int rc = obem_fieldmap_build_nodes(c, sigma, (cudaStream_t)stream);
    if (rc != OBEM_OK) {
        free_dev(c->fm.nodes);
        memset(&c->fm, 0, sizeof c->fm);
    }
    return rc;
}

extern "C" int obem_fieldmap_eval(obem_ctx *c, const float *points, int32_t n, float *E_out, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (!c->fm.nodes) return obem_fail(c, OBEM_ERR_STATE, "field map: call obem_fieldmap_build first");
    if (n < 0) return obem_fail(c, OBEM_ERR_ARG, "field map: negative count");
    if (n == 0) return OBEM_OK;
    if (!points || !E_out) return obem_fail(c, OBEM_ERR_ARG, "field map: null points or E_out");
    if (((uintptr_t)points | (uintptr_t)E_out) & 15)
        return obem_fail(c, OBEM_ERR_ARG, "field map: arrays must be 16-byte aligned");
    return obem_fieldmap_interp(c, (const float4 *)points, NULL, n, (float4 *)E_out, make_float3(0.f, 0.f, 0.f),
                                (cudaStream_t)stream);
}

extern "C" int obem_step(obem_ctx *c, const obem_state *st, const float *E_in, uint32_t step,
                         obem_step_stats *stats, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    if (!c->gas_loaded) return obem_fail(c, OBEM_ERR_STATE, "step: call obem_gas_load first");
    if (!st || !stats) return obem_fail(c, OBEM_ERR_ARG, "step: null state or stats");
    if (!st->pos_q || !st->vel || !st->id || !st->birth || !st->species || !st->n || !st->next_id)
        return obem_fail(c, OBEM_ERR_ARG, "step: null state array");
    if (st->capacity < 1 || st->capacity > c->cap)
        return obem_fail(c, OBEM_ERR_ARG, "step: state capacity %d outside 1..%d", st->capacity, c->cap);
    if (((uintptr_t)st->pos_q | (uintptr_t)st->vel | (uintptr_t)E_in) & 15)
        return obem_fail(c, OBEM_ERR_ARG, "step: pos_q / vel / E_in must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const float4 *E = (const float4 *)E_in;
    cudaEvent_t *ev = NULL;
    if (c->prof_on) {
        ev = c->prof_ev + OBEM_PROF_EV * (c->prof_n % OBEM_PROF_MAX);
        if (c->prof_n < OBEM_PROF_MAX) c->prof_n++;
        cudaEventRecord(ev[0], s);
        cudaEventRecord(ev[4], s);
        cudaEventRecord(ev[5], s);
    }
    const int want_map = (c->cfg.flags & OBEM_STEP_FIELD_MAP) != 0;
    if (want_map && !E && !c->fm.nodes)
        return obem_fail(c, OBEM_ERR_STATE, "step: OBEM_STEP_FIELD_MAP without obem_fieldmap_build");
    int want_cells = !want_map && (c->cfg.flags & OBEM_STEP_CELL_FIELD) && c->sigma_valid;
    int want_nbody = (c->cfg.flags & OBEM_STEP_SPACE_CHARGE) != 0;
    if (!E) {
        const float3 e_ext = make_float3((float)c->cfg.e_ext[0], (float)c->cfg.e_ext[1], (float)c->cfg.e_ext[2]);
        if (want_map) {
            // cell field (+ e_ext) from the map; the all-pairs sum adds to it
            int rc = obem_fieldmap_interp(c, (const float4 *)st->pos_q, st->n, st->capacity, c->s_E, e_ext, s);
            if (rc != OBEM_OK) return rc;
            if (c->prof_on) c->launches++;
        }
        FieldLaunch L;
        memset(&L, 0, sizeof L);
        L.targets = (const float4 *)st->pos_q;
        L.nt_dev = st->n;
        L.nt = st->capacity;
        L.sources = want_nbody ? (const float4 *)st->pos_q : NULL;
        L.ns_dev = st->n;
        L.ns = st->capacity;
        L.self_exclude = 1;
        L.eps2 = (float)(c->cfg.softening * c->cfg.softening);
        L.sigma = want_cells ? c->d_sigma : NULL;
        L.panels = panels_of(c);
        L.perm = want_cells ? c->s_perm : NULL;
        L.blocks = want_cells ? c->s_blocks : NULL;
        L.nblocks = want_cells ? c->s_nblocks : NULL;
        L.E_out = c->s_E;
        L.e_ext = e_ext;
        L.add_init = want_map;
        L.nn_grid = (c->cfg.flags & OBEM_STEP_NBODY_NN) ? (c->cfg.nn_grid > 0 ? c->cfg.nn_grid : 16) : 0;
        L.want_v = 0;
        if (ev && c->prof_on == 1) L.counters = c->d_counters;     // tier counters (counting kernels)
        L.events = ev;
        int rc = obem_launch_field(c, L, st->capacity, s);
        if (rc != OBEM_OK) return rc;
        E = c->s_E;
    } else if (ev) {
        cudaEventRecord(ev[1], s);
        cudaEventRecord(ev[2], s);
    }
    int rc = obem_launch_step(c, st, E, step, stats, s);
    if (ev) cudaEventRecord(ev[3], s);
    return rc;
}
