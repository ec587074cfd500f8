// A batch of independent chambers stepped together (many small chambers
// with uneven charge counts, e.g. a sweep over gaps and fields of the
// parallel-plate counter of Sec. 4.1).  One concatenated charge state holds
// every chamber in a segment of its own; every stage of the step (cell field,
// all-pairs field, tracking passes) is one launch for all chambers, the
// all-pairs stage a persistent kernel over every chamber's work units, and the
// step index lives on the device, so the whole step can be captured once in a
// CUDA graph and replayed.  A small autotuner picks the cell-kernel block size
// by timing the field on the batch's own charges.
#include <vector>

#include "obem_internal.cuh"

struct obem_batch {
    obem_ctx *ctx;               // gas, dt, softening, beta, trial cap, flags, error text
    int nb, slots;
    std::vector<int32_t> seg_off;          // [nb + 1]
    std::vector<int> np;                   // cells per chamber
    std::vector<std::vector<double>> tri;  // FP64 vertices per chamber
    std::vector<std::vector<float>> sig;   // densities per chamber
    int cells_dirty;
    int cut;                               // cell-kernel block size
    // device tables
    int32_t *d_seg_off, *d_blk_cham, *d_slot_cham;
    ChamberP *d_cham;
    StepCtl *d_ctl;
    int32_t *d_abort;
    // cells of every chamber, concatenated
    int np_total;
    float4 *d_c_a, *d_g0_h, *d_g1, *d_g2, *d_nrm, *d_c_lo;
    double *d_v64, *d_geo64;
    float *d_sigma;
    int2 *d_cham_pan;
    // field scratch
    float4 *d_E;
    int2 *d_blocks;
    int32_t *d_block_cham, *d_nblocks;
    float *d_jpart, *d_ipart;
    long long *d_joff, *d_ioff;
    float4 *d_sorted;
    int32_t *d_perm, *d_bcnt, *d_negtot, *d_uoff;
    int *d_counter;
    float *d_tileq;
    int sym_grid;
    BtScratch W;
    // captured step
    cudaGraphExec_t graph;
    cudaStream_t cap_stream;
    const void *graph_key[9];
};

static void bfree(void *p)
{
    if (p) cudaFree(p);
}

static void free_cells(obem_batch *b)
{
    bfree(b->d_c_a); bfree(b->d_g0_h); bfree(b->d_g1); bfree(b->d_g2); bfree(b->d_nrm); bfree(b->d_c_lo);
    bfree(b->d_v64); bfree(b->d_geo64); bfree(b->d_sigma);
    b->d_c_a = b->d_g0_h = b->d_g1 = b->d_g2 = b->d_nrm = b->d_c_lo = NULL;
    b->d_v64 = b->d_geo64 = NULL;
    b->d_sigma = NULL;
    b->np_total = 0;
}

extern "C" void obem_batch_destroy(obem_batch *b)
{
    if (!b) return;
    free_cells(b);
    bfree(b->d_seg_off); bfree(b->d_blk_cham); bfree(b->d_slot_cham); bfree(b->d_cham); bfree(b->d_ctl);
    bfree(b->d_abort); bfree(b->d_cham_pan); bfree(b->d_E); bfree(b->d_blocks); bfree(b->d_block_cham);
    bfree(b->d_nblocks); bfree(b->d_jpart); bfree(b->d_ipart); bfree(b->d_joff); bfree(b->d_ioff);
    bfree(b->d_sorted); bfree(b->d_perm); bfree(b->d_bcnt); bfree(b->d_negtot); bfree(b->d_uoff);
    bfree(b->d_counter); bfree(b->d_tileq);
    BtScratch &W = b->W;
    bfree(W.prop); bfree(W.ionkey); bfree(W.keep); bfree(W.nsp); bfree(W.blk); bfree(W.o_pos); bfree(W.o_vel);
    bfree(W.o_id); bfree(W.o_birth); bfree(W.o_sp); bfree(W.ph_bucket); bfree(W.ph_count); bfree(W.ph_start);
    bfree(W.ph_cursor); bfree(W.ph_sorted); bfree(W.ph_bsum); bfree(W.mpart);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

#define OBEM_PH_BUCKETS (1 << 20)

extern "C" int obem_batch_create(obem_batch **out, obem_ctx *ctx, int32_t n_chambers, const int32_t *capacity,
                                 const double *z_lo, const double *z_hi, const uint64_t *seed)
{
    if (!out || !ctx) return OBEM_ERR_ARG;
    *out = NULL;
    if (n_chambers < 1 || n_chambers > 65536 || !capacity || !z_lo || !z_hi || !seed)
        return obem_fail(ctx, OBEM_ERR_ARG, "batch: need 1..65536 chambers and their capacity, planes, seeds");
    if (!ctx->gas_loaded) return obem_fail(ctx, OBEM_ERR_STATE, "batch: load the gas into the context first");
    const int allowed = OBEM_STEP_SPACE_CHARGE | OBEM_STEP_CELL_FIELD | OBEM_STEP_PROB_COLLISION;
    if (ctx->cfg.flags & ~allowed)
        return obem_fail(ctx, OBEM_ERR_ARG, "batch: only SPACE_CHARGE, CELL_FIELD and PROB_COLLISION steps");
    long long slots = 0;
    std::vector<int32_t> off(n_chambers + 1);
    for (int c = 0; c < n_chambers; ++c) {
        if (capacity[c] < 1 || !(z_lo[c] < z_hi[c]))
            return obem_fail(ctx, OBEM_ERR_ARG, "batch: chamber %d needs capacity >= 1 and z_lo < z_hi", c);
        off[c] = (int32_t)slots;
        slots += ((long long)capacity[c] + OBEM_SEG_ALIGN - 1) / OBEM_SEG_ALIGN * OBEM_SEG_ALIGN;
        if (slots > 0x40000000ll) return obem_fail(ctx, OBEM_ERR_ARG, "batch: more than 2^30 slots");
    }
    off[n_chambers] = (int32_t)slots;
    obem_batch *b = new obem_batch();
    b->ctx = ctx;
    b->nb = n_chambers;
    b->slots = (int)slots;
    b->seg_off = off;
    b->np.assign(n_chambers, 0);
    b->tri.resize(n_chambers);
    b->sig.resize(n_chambers);
    b->cut = 512;
    const int nb = n_chambers, S = b->slots;
    std::vector<int32_t> blk_cham(S / 256), slot_cham(S / OBEM_SEG_ALIGN);
    std::vector<ChamberP> cham(nb);
    std::vector<long long> joff(nb), ioff(nb);
    long long jt = 0, it = 0;
    int max_blocks = 0;
    for (int c = 0; c < nb; ++c) {
        for (int k = off[c] / 256; k < off[c + 1] / 256; ++k) blk_cham[k] = c;
        for (int k = off[c] / OBEM_SEG_ALIGN; k < off[c + 1] / OBEM_SEG_ALIGN; ++k) slot_cham[k] = c;
        cham[c].seed_lo = (uint32_t)(seed[c] & 0xFFFFFFFFu);
        cham[c].seed_hi = (uint32_t)(seed[c] >> 32);
        cham[c].z_lo = (float)z_lo[c];
        cham[c].z_hi = (float)z_hi[c];
        // a chamber may fill its whole segment: everything is sized by its length
        const int seg = off[c + 1] - off[c];
        size_t ipf;
        const size_t jpf = obem_sym_sizes(seg, &ipf);
        joff[c] = jt;
        ioff[c] = it;
        jt += (long long)jpf;
        it += (long long)ipf;
        max_blocks += seg / 32;                    // enough for the smallest block size
    }
    int rc = OBEM_OK;
#define BALLOC(p, bytes)                                                                          \
    do {                                                                                          \
        if (rc == OBEM_OK && cudaMalloc((void **)&(p), (size_t)(bytes)) != cudaSuccess)           \
            rc = obem_fail(ctx, OBEM_ERR_CUDA, "batch: allocation of %zu bytes failed", (size_t)(bytes)); \
    } while (0)
#define BUP(p, src, bytes)                                                                        \
    do {                                                                                          \
        BALLOC(p, bytes);                                                                         \
        if (rc == OBEM_OK && cudaMemcpy((p), (src), (size_t)(bytes), cudaMemcpyHostToDevice) != cudaSuccess) \
            rc = obem_fail(ctx, OBEM_ERR_CUDA, "batch: upload failed");                           \
    } while (0)
    BUP(b->d_seg_off, off.data(), sizeof(int32_t) * (nb + 1));
    BUP(b->d_blk_cham, blk_cham.data(), sizeof(int32_t) * blk_cham.size());
    BUP(b->d_slot_cham, slot_cham.data(), sizeof(int32_t) * slot_cham.size());
    BUP(b->d_cham, cham.data(), sizeof(ChamberP) * nb);
    BUP(b->d_joff, joff.data(), sizeof(long long) * nb);
    BUP(b->d_ioff, ioff.data(), sizeof(long long) * nb);
    BALLOC(b->d_ctl, sizeof(StepCtl) * nb);
    BALLOC(b->d_abort, sizeof(int32_t));
    BALLOC(b->d_cham_pan, sizeof(int2) * nb);
    BALLOC(b->d_E, sizeof(float4) * S);
    BALLOC(b->d_blocks, sizeof(int2) * max_blocks);
    BALLOC(b->d_block_cham, sizeof(int32_t) * max_blocks);
    BALLOC(b->d_nblocks, sizeof(int32_t));
    BALLOC(b->d_jpart, sizeof(float) * jt);
    BALLOC(b->d_ipart, sizeof(float) * it);
    BALLOC(b->d_sorted, sizeof(float4) * S);
    BALLOC(b->d_perm, sizeof(int32_t) * S);
    BALLOC(b->d_bcnt, sizeof(int32_t) * (S / OBEM_SEG_ALIGN + 1));
    BALLOC(b->d_negtot, sizeof(int32_t) * nb);
    BALLOC(b->d_uoff, sizeof(int32_t) * (nb + 1));
    BALLOC(b->d_counter, sizeof(int));
    BALLOC(b->d_tileq, sizeof(float) * (S / OBEM_SEG_ALIGN));
    BtScratch &W = b->W;
    BALLOC(W.prop, sizeof(unsigned long long) * S);
    BALLOC(W.ionkey, sizeof(unsigned long long) * S);
    BALLOC(W.keep, sizeof(int32_t) * S);
    BALLOC(W.nsp, sizeof(int32_t) * S);
    BALLOC(W.blk, sizeof(int32_t) * 2 * (S / 256));
    BALLOC(W.o_pos, sizeof(float4) * S);
    BALLOC(W.o_vel, sizeof(float4) * S);
    BALLOC(W.o_id, sizeof(uint32_t) * S);
    BALLOC(W.o_birth, sizeof(uint32_t) * S);
    BALLOC(W.o_sp, S);
    BALLOC(W.ph_bucket, sizeof(int32_t) * S);
    BALLOC(W.ph_count, sizeof(int32_t) * OBEM_PH_BUCKETS);
    BALLOC(W.ph_start, sizeof(int32_t) * (OBEM_PH_BUCKETS + 1));
    BALLOC(W.ph_cursor, sizeof(int32_t) * OBEM_PH_BUCKETS);
    BALLOC(W.ph_sorted, sizeof(int32_t) * S);
    BALLOC(W.ph_bsum, sizeof(int32_t) * (OBEM_PH_BUCKETS / 1024 + 1));
    BALLOC(W.mpart, sizeof(double) * 13 * (S / 256));
    if (rc == OBEM_OK) {
        std::vector<int2> pan(nb, make_int2(0, 0));
        if (cudaMemcpy(b->d_cham_pan, pan.data(), sizeof(int2) * nb, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = obem_fail(ctx, OBEM_ERR_CUDA, "batch: upload failed");
    }
    if (rc == OBEM_OK) {
        b->sym_grid = obem_sym_grid(ctx->device);
        if (b->sym_grid <= 0) rc = obem_fail(ctx, OBEM_ERR_CUDA, "batch: no occupancy for the all-pairs kernel");
    }
    if (rc != OBEM_OK) {
        obem_batch_destroy(b);
        return rc;
    }
    *out = b;
    return OBEM_OK;
}

extern "C" int obem_batch_layout(const obem_batch *b, int64_t *seg_off)
{
    if (!b || !seg_off) return OBEM_ERR_ARG;
    for (int c = 0; c <= b->nb; ++c) seg_off[c] = b->seg_off[c];
    return OBEM_OK;
}

extern "C" int obem_batch_cells(obem_batch *b, int32_t chamber, int32_t n_cells, const double *tri_xyz,
                                const float *sigma)
{
    if (!b) return OBEM_ERR_ARG;
    if (chamber < 0 || chamber >= b->nb) return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: no chamber %d", chamber);
    if (n_cells < 0 || n_cells > 200000 || (n_cells > 0 && (!tri_xyz || !sigma)))
        return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: cells of chamber %d: 0..200000 cells, vertices, densities",
                         chamber);
    b->np[chamber] = n_cells;
    b->tri[chamber].assign(tri_xyz, tri_xyz + 9 * (size_t)n_cells);
    b->sig[chamber].assign(sigma, sigma + n_cells);
    b->cells_dirty = 1;
    return OBEM_OK;
}

// concatenate the chambers' cells and upload them (synchronous; not while a
// stream is being captured)
static int upload_cells(obem_batch *b)
{
    obem_ctx *ctx = b->ctx;
    free_cells(b);
    long long tot = 0;
    std::vector<int2> pan(b->nb);
    for (int c = 0; c < b->nb; ++c) {
        pan[c] = make_int2((int)tot, b->np[c]);
        tot += b->np[c];
    }
    if (tot > 0x7fffffff / 9) return obem_fail(ctx, OBEM_ERR_ARG, "batch: too many cells");
    const int np = (int)tot;
    int rc = OBEM_OK;
    if (np > 0) {
        std::vector<double> v64(9 * (size_t)np);
        std::vector<float> sg(np);
        for (int c = 0; c < b->nb; ++c) {
            std::copy(b->tri[c].begin(), b->tri[c].end(), v64.begin() + 9 * (size_t)pan[c].x);
            std::copy(b->sig[c].begin(), b->sig[c].end(), sg.begin() + pan[c].x);
        }
        std::vector<float4> ca(np), g0(np), g1(np), g2(np), nr(np), cl(np);
        const int bad = obem_cell_layout(v64.data(), NULL, np, ca.data(), g0.data(), g1.data(), g2.data(),
                                         nr.data(), cl.data());
        if (bad >= 0) return obem_fail(ctx, OBEM_ERR_ARG, "batch: cell %d (of all chambers) is degenerate", bad);
        const size_t f4 = sizeof(float4) * np;
        BUP(b->d_c_a, ca.data(), f4);
        BUP(b->d_g0_h, g0.data(), f4);
        BUP(b->d_g1, g1.data(), f4);
        BUP(b->d_g2, g2.data(), f4);
        BUP(b->d_nrm, nr.data(), f4);
        BUP(b->d_c_lo, cl.data(), f4);
        BUP(b->d_v64, v64.data(), sizeof(double) * 9 * (size_t)np);
        std::vector<double> geo((size_t)OBEM_GEO64 * np);
        obem_cell_geo64(v64.data(), np, geo.data());
        BUP(b->d_geo64, geo.data(), sizeof(double) * geo.size());
        BUP(b->d_sigma, sg.data(), sizeof(float) * np);
    }
    if (rc == OBEM_OK &&
        cudaMemcpy(b->d_cham_pan, pan.data(), sizeof(int2) * b->nb, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = obem_fail(ctx, OBEM_ERR_CUDA, "batch: upload failed");
    if (rc != OBEM_OK) {
        free_cells(b);
        return rc;
    }
    b->np_total = np;
    b->cells_dirty = 0;
    return OBEM_OK;
}
#undef BUP
#undef BALLOC

static int check_state(obem_batch *b, const obem_state *st)
{
    if (!st || !st->pos_q || !st->vel || !st->id || !st->birth || !st->species || !st->n || !st->next_id)
        return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: state with a null array");
    if (st->capacity != b->slots)
        return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: state capacity %d is not the batch's %d slots", st->capacity,
                         b->slots);
    if (((uintptr_t)st->pos_q | (uintptr_t)st->vel) & 15)
        return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: pos_q / vel must be 16-byte aligned");
    return OBEM_OK;
}

static int prepare(obem_batch *b, cudaStream_t s)
{
    if (!b->cells_dirty) return OBEM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return obem_fail(b->ctx, OBEM_ERR_STATE, "batch: cells changed; step once outside stream capture");
    return upload_cells(b);
}

static FieldBatch field_args(obem_batch *b, const obem_state *st)
{
    obem_ctx *ctx = b->ctx;
    FieldBatch F;
    memset(&F, 0, sizeof F);
    F.nb = b->nb;
    F.slots = b->slots;
    F.cut = b->cut;
    F.max_blocks = 0;
    for (int c = 0; c < b->nb; ++c)
        F.max_blocks += (b->seg_off[c + 1] - b->seg_off[c] + b->cut - 1) / b->cut;
    F.cells = (ctx->cfg.flags & OBEM_STEP_CELL_FIELD) && b->np_total > 0;
    F.charges = (ctx->cfg.flags & OBEM_STEP_SPACE_CHARGE) != 0;
    F.eps2 = (float)(ctx->cfg.softening * ctx->cfg.softening);
    F.e_ext = make_float3((float)ctx->cfg.e_ext[0], (float)ctx->cfg.e_ext[1], (float)ctx->cfg.e_ext[2]);
    F.panels.c_a = b->d_c_a;
    F.panels.g0_h = b->d_g0_h;
    F.panels.g1 = b->d_g1;
    F.panels.g2 = b->d_g2;
    F.panels.nrm = b->d_nrm;
    F.panels.c_lo = b->d_c_lo;
    F.panels.v64 = b->d_v64;
    F.panels.geo = b->d_geo64;
    F.panels.np = b->np_total;
    F.sigma = b->d_sigma;
    F.cham_pan = b->d_cham_pan;
    F.blocks = b->d_blocks;
    F.block_cham = b->d_block_cham;
    F.nblocks = b->d_nblocks;
    F.sym.nb = b->nb;
    F.sym.seg_off = b->d_seg_off;
    F.sym.n = st->n;
    F.sym.slot_cham = b->d_slot_cham;
    F.sym.joff = b->d_joff;
    F.sym.ioff = b->d_ioff;
    F.sym.uoff = b->d_uoff;
    F.sym.negtot = b->d_negtot;
    F.jpart = b->d_jpart;
    F.ipart = b->d_ipart;
    F.sorted = b->d_sorted;
    F.perm = b->d_perm;
    F.bcnt = b->d_bcnt;
    F.tileq = b->d_tileq;
    F.counter = b->d_counter;
    F.sym_grid = b->sym_grid;
    return F;
}

extern "C" int obem_batch_field_eval(obem_batch *b, const obem_state *st, float *E_out, obem_stream stream)
{
    if (!b) return OBEM_ERR_ARG;
    int rc = check_state(b, st);
    if (rc != OBEM_OK) return rc;
    if (!E_out || ((uintptr_t)E_out & 15)) return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: E_out null or unaligned");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = prepare(b, s)) != OBEM_OK) return rc;
    const FieldBatch F = field_args(b, st);
    return obem_launch_field_batch(b->ctx, F, (const float4 *)st->pos_q, (float4 *)E_out, s);
}

extern "C" int obem_batch_step(obem_batch *b, const obem_state *st, const float *E_in, uint32_t *step,
                               obem_step_stats *stats, obem_stream stream)
{
    if (!b) return OBEM_ERR_ARG;
    int rc = check_state(b, st);
    if (rc != OBEM_OK) return rc;
    if (!step || !stats) return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: step index and stats are required");
    if ((uintptr_t)E_in & 15) return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: E_in must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = prepare(b, s)) != OBEM_OK) return rc;
    const float4 *E = (const float4 *)E_in;
    if (!E) {
        const FieldBatch F = field_args(b, st);
        if ((rc = obem_launch_field_batch(b->ctx, F, (const float4 *)st->pos_q, b->d_E, s)) != OBEM_OK) return rc;
        E = b->d_E;
    }
    StepBatch B;
    B.nb = b->nb;
    B.seg_off = b->d_seg_off;
    B.blk_cham = b->d_blk_cham;
    B.n = st->n;
    B.next_id = st->next_id;
    B.cham = b->d_cham;
    B.stats = stats;
    B.ctl = b->d_ctl;
    B.abort = b->d_abort;
    B.step = step;
    return obem_launch_step_batch(b->ctx, st, B, b->W, E, s);
}

// The fused step captured once (per state, step index and stats arrays) and
// replayed: every replay is one step of every chamber.
extern "C" int obem_batch_step_graph(obem_batch *b, const obem_state *st, uint32_t *step, obem_step_stats *stats,
                                     obem_stream stream)
{
    if (!b) return OBEM_ERR_ARG;
    int rc = check_state(b, st);
    if (rc != OBEM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = prepare(b, s)) != OBEM_OK) return rc;
    const void *key[9] = {st->pos_q, st->vel, st->id, st->birth, st->species, st->n, st->next_id, step, stats};
    bool hit = b->graph != NULL;
    for (int k = 0; k < 9 && hit; ++k) hit = key[k] == b->graph_key[k];
    if (!hit) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = NULL;
        }
        // captured on a private stream (nothing runs there); launched on s
        if (!b->cap_stream) OBEM_CUDA(b->ctx, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        OBEM_CUDA(b->ctx, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = obem_batch_step(b, st, NULL, step, stats, (obem_stream)b->cap_stream);
        cudaGraph_t g = NULL;
        const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (rc != OBEM_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess || !g)
            return obem_fail(b->ctx, OBEM_ERR_CUDA, "batch: capture failed: %s", cudaGetErrorString(e));
        const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            b->graph = NULL;
            return obem_fail(b->ctx, OBEM_ERR_CUDA, "batch: graph instantiation failed: %s", cudaGetErrorString(ei));
        }
        for (int k = 0; k < 9; ++k) b->graph_key[k] = key[k];
    }
    OBEM_CUDA(b->ctx, cudaGraphLaunch(b->graph, s));
    return OBEM_OK;
}

// Autotuner: the cell-kernel block size (targets per block: smaller blocks
// have tighter boxes, so fewer near cells and cheaper tiers, but repeat the
// per-block tiering of every cell more often) is picked by timing the field on
// the batch's current charges, best of `reps` runs per candidate.  The chosen
// size stays in force (and changes the field only by the rounding of the
// tiered sums).  out: host [4]: chosen size, its time (ms), the time of 512.
extern "C" int obem_batch_autotune(obem_batch *b, const obem_state *st, int32_t reps, double *out,
                                   obem_stream stream)
{
    if (!b || !out) return OBEM_ERR_ARG;
    int rc = check_state(b, st);
    if (rc != OBEM_OK) return rc;
    if (reps < 1 || reps > 100) return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: reps outside 1..100");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = prepare(b, s)) != OBEM_OK) return rc;
    const int cand[3] = {128, 256, 512};
    double best = 1e300, t512 = 0.0;
    int best_cut = 512;
    cudaEvent_t e0, e1;
    OBEM_CUDA(b->ctx, cudaEventCreate(&e0));
    OBEM_CUDA(b->ctx, cudaEventCreate(&e1));
    for (int k = 0; k < 3 && rc == OBEM_OK; ++k) {
        b->cut = cand[k];
        const FieldBatch F = field_args(b, st);
        double tmin = 1e300;
        for (int r = 0; r < reps + 1 && rc == OBEM_OK; ++r) {       // first run warms up
            cudaEventRecord(e0, s);
            rc = obem_launch_field_batch(b->ctx, F, (const float4 *)st->pos_q, b->d_E, s);
            cudaEventRecord(e1, s);
            if (rc != OBEM_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = obem_fail(b->ctx, OBEM_ERR_CUDA, "batch: autotune run failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms < tmin) tmin = ms;
        }
        if (cand[k] == 512) t512 = tmin;
        if (tmin < best) { best = tmin; best_cut = cand[k]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cut = best_cut;
    if (b->graph) {                  // the captured step used the old size
        cudaGraphExecDestroy(b->graph);
        b->graph = NULL;
    }
    if (rc != OBEM_OK) return rc;
    out[0] = best_cut;
    out[1] = best;
    out[2] = t512;
    out[3] = 0.0;
    return OBEM_OK;
}

extern "C" int obem_batch_set_block(obem_batch *b, int32_t cut)
{
    if (!b) return OBEM_ERR_ARG;
    if (cut < 32 || cut > 512) return obem_fail(b->ctx, OBEM_ERR_ARG, "batch: block size outside 32..512");
    b->cut = cut;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = NULL;
    }
    return OBEM_OK;
}
