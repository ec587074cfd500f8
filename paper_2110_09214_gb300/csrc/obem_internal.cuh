// Internal declarations shared by the translation units of libobem.
// Not part of the public ABI (include/obem.h is).
#pragma once

#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/obem.h"

// ---------------------------------------------------------------- constants
// CODATA 2018 (SI)
#define OBEM_QE 1.602176634e-19
#define OBEM_ME 9.1093837015e-31
#define OBEM_EPS0 8.8541878128e-12
#define OBEM_KB 1.380649e-23
#define OBEM_AMU 1.66053906660e-27
#define OBEM_PI 3.14159265358979323846
#define OBEM_KC (1.0 / (4.0 * OBEM_PI * OBEM_EPS0))

#define OBEM_MAX_PROC 32
#define OBEM_MAX_TRIALS 256
#define OBEM_NCOUNTERS 7      // evaluation counters of the profiling variants of the field kernels

// ---------------------------------------------------------------- gas constants
// Everything the step kernels need, passed by value.  The float members are
// derived in FP64 on the host and rounded once.
struct GasDev {
    const float *egrid;   // [n_e]
    const float *xs;      // [n_proc][n_e]
    int n_proc, n_e;
    int kind[OBEM_MAX_PROC];
    int mode[OBEM_MAX_PROC];
    float thr[OBEM_MAX_PROC];
    float nuc[OBEM_MAX_PROC];
    float dt, nu_max_e, nu_ion, half_nu_ion, E_therm, v_th_ion;
    float qm[3];
    float K_e, two_m_over_M, KCE, N, z_lo, z_hi, rc2;
    float ion_thr;
    int recomb_on;
    uint32_t seed_lo, seed_hi;
    int trial_cap;
    int coll_mode;        // 0: null-collision trials; 1: per-step probability (OBEM_STEP_PROB_COLLISION)
    // cells absorbing the charges crossing them (OBEM_STEP_SURFACE_HITS)
    int hit_on;
    const float *tri9;    // binary32 vertices [np][9]
    const int32_t *hstart, *htri;   // uniform grid over the cells: CSR lists of cells per grid cell
    float hlo[3], hinv;
    int hdim[3];
};

// Cell geometry in the layout of the field kernels (structure of arrays).
//   c_a  = (cx, cy, cz, k_C * area)
//   g0_h = (v0 - c, h^2)      h = longest edge
//   g1   = (v1 - c, 0)
//   g2   = (v2 - c, 0)
//   v64  = FP64 vertices [np][9] for the near-field closed form
//   nrm  = (nx, ny, nz, kind)
//   c_lo = centroid - float(centroid), so that (c_a.xyz + c_lo.xyz) carries the
//          centroid to ~2^-48 relative (differences to nearby targets stay exact)
struct PanelsDev {
    const float4 *c_a, *g0_h, *g1, *g2, *nrm, *c_lo;
    const double *v64;
    // FP64 geometry of each cell for the closed form, OBEM_GEO64 doubles per
    // cell (unit normal, twice the area, unit edge vectors and in-plane edge
    // normals), or NULL (then computed per evaluation)
    const double *geo;
    int np;
};
#define OBEM_GEO64 24

// Static field map: cell field on a regular grid (valid nx x ny x nz nodes,
// stored padded to px x py x pz in bricks of 8^3), node (i, j, k) at
// lo + (i, j, k) * step.
struct FieldMapDev {
    float4 *nodes;
    int nx, ny, nz, px, py, pz;
    double lo[3], step[3];
};

// Device-resident control block of one obem_step call.
struct StepCtl {
    int32_t abort;        // non-zero: do not commit
    int32_t n_keep;       // survivors
    int32_t n_spawn;      // spawned pairs
    int32_t trial_overflow;
};

// What differs between the chambers of a batch in the tracking step: Philox
// key and electrode planes
struct ChamberP {
    uint32_t seed_lo, seed_hi;
    float z_lo, z_hi;
};

// A batch of chambers as the batched step kernels see it (see SymBatch for the
// slot layout; blocks of 256 slots belong to one chamber)
struct StepBatch {
    int nb;
    const int32_t *seg_off;      // [nb + 1]
    const int32_t *blk_cham;     // [seg_off[nb] / 256]
    int32_t *n;                  // [nb] live charges
    uint32_t *next_id;           // [nb]
    const ChamberP *cham;        // [nb]
    obem_step_stats *stats;      // [nb]
    StepCtl *ctl;                // [nb]
    int32_t *abort;              // [1]
    uint32_t *step;              // [1] step index, advanced when the batch commits
};

// scratch of the batched step, sized for the batch's slots
struct BtScratch {
    unsigned long long *prop, *ionkey;
    int32_t *keep, *nsp, *blk;
    float4 *o_pos, *o_vel;
    uint32_t *o_id, *o_birth;
    uint8_t *o_sp;
    int32_t *ph_bucket, *ph_count, *ph_start, *ph_cursor, *ph_sorted, *ph_bsum;
    double *mpart;           // per-block partial moments (13 per block of 256 slots)
};

struct obem_ctx {
    obem_config cfg;
    char err[512];
    int device;
    // gas
    int gas_loaded;
    GasDev gas;
    float *d_egrid, *d_xs;
    float gas_thr_ioni;
    double gas_T, gas_N, gas_M_amu, gas_nu_ion;
    // mesh
    int np, n_groups;
    int *h_kind, *h_group;
    double *h_tri, *h_em, *h_ep;
    float4 *d_c_a, *d_g0_h, *d_g1, *d_g2, *d_nrm, *d_c_lo;
    double *d_v64;
    double *d_geo64;         // [np][OBEM_GEO64] closed-form geometry
    int *d_kind, *d_group;
    float bbox_lo[3], bbox_hi[3];   // of the cell vertices (target binning grid)
    // BEM
    int nsys, nsys_alloc; // size of the system held (np after obem_bem_assemble) and of its buffers
    float *d_A;          // equilibrated matrix, row-major [nsys][nsys]
    float *d_LU;         // LU factors (row-major, unit lower L below the diagonal)
    int *d_piv;          // row swaps of the factorisation
    double *d_rowscale;  // 1 / max |A_ij| per row
    double *d_work64;    // 4 * np doubles
    float *d_work32;     // 2 * np floats
    int *d_flag;         // device status of the LU (singular / timeout)
    float *d_panel;      // exchange buffers of the pivoting panel kernel
    int *d_trsv;         // one-launch triangular solves: block flags, ticket counter, status
    int trsv_epoch;      // flag value of the last triangular-solve launch
    float *d_dinv;       // inverses of the diagonal blocks of L and U, [nbk][2][TS_R][TS_R]
    int *d_perm;         // row permutation of the factorisation: (P b)[i] = b[d_perm[i]]
    int factored;
    double factor_ms;
    double a_norm_inf;
    float *d_sigma;      // current sigma [np]
    double *d_infl;      // [np][4] charge sums of the influence right-hand side (obem_influence_rhs)
    double *d_epsd;      // [np] eps_plus - eps_minus of the dielectric cells (0 on electrode cells)
    void *d_ib;          // scratch of the influence pass (binned charges), ib_bytes
    size_t ib_bytes;
    int sigma_valid;
    unsigned long long sigma_ver;   // bumped whenever d_sigma is rewritten
    // far-cell groups (OBEM_STEP_CELL_GROUPS; ngrp == 0: not built)
    int ngrp;
    int32_t *d_grp_perm;
    float4 *d_grp_cr;
    float *d_grp_h2min;
    float4 *d_grp_u;
    float *d_grp_q;
    double *d_grp_c64;   // [ngrp][4] centre and radius as the binary32 values, in FP64
    double *d_grp_v;     // [OBEM_GRP_CHECK][3] unit directions of the check points
    double *d_grp_pinv;  // [OBEM_GRP_M][OBEM_GRP_CHECK] least-squares fit for a unit radius
    const float *grp_fit_sigma;     // sigma the charges in d_grp_q were fitted to (d_sigma only)
    unsigned long long grp_fit_ver; // and its version
    cublasHandle_t cublas;
    // BF16 operand scratch of the tensor-core LU updates (lu_tc.cu)
    void *tc_a, *tc_b;
    size_t tc_a_bytes, tc_b_bytes;
    // step scratch (capacity-sized)
    float4 *s_E;
    unsigned long long *s_prop, *s_ionkey;
    int32_t *s_keep, *s_nsp;
    int32_t *s_blk;       // per-block sums / offsets (2 * max_blocks)
    double *s_mpart;      // per-block partial moments (13 * max_blocks)
    StepCtl *s_ctl;
    float4 *o_pos, *o_vel;
    uint32_t *o_id, *o_birth;
    uint8_t *o_sp;
    int cap;
    // target binning (Morton order of a 64^3 grid) for the cell kernels
    uint32_t *s_code;
    int32_t *s_perm;
    int32_t *s_hist;
    int2 *s_blocks;        // cell-kernel blocks: (first sorted target, count)
    int32_t *s_nblocks;    // [1] number of blocks, [2..] scan scratch
    // symmetric all-pairs kernel (targets == sources): per-item source-side and
    // per-unit target-side partial sums, work counter, persistent grid; NULL
    // when they did not fit the memory budget (the one-sided kernel runs)
    float *sym_jpart, *sym_ipart;   // one pass of diagonals (field.cu SymPass)
    double *sym_acc;                 // [capacity][4] FP64 sums carried between passes
    // partner search: hash-bucket counts / starts / cursors, bucket of each
    // charge, cations sorted by bucket
    int32_t *ph_count, *ph_start, *ph_cursor, *ph_bucket, *ph_sorted, *ph_bsum;
    // static field map (nodes == NULL until obem_fieldmap_build)
    FieldMapDev fm;
    // charging-up: binary32 vertices, uniform grid over the cells, cell
    // areas, charges deposited per cell (units of e) and per-step hits
    float *d_tri9;
    int32_t *d_hstart, *d_htri;
    float h_hlo[3], h_hinv;
    int h_hdim[3];
    double *d_area;
    long long *d_deposit;
    int32_t *s_hit;
    // approximate N-body: bounding box, cell of each charge, cell counts /
    // starts / cursors, charges sorted by cell, per-cell charge centres
    int *nn_bbox;
    int32_t *nn_cell, *nn_sorted, *nn_count, *nn_start, *nn_cursor;
    float4 *nn_agg;
    int *sym_counter;
    uint32_t *s_tk;          // stable bin sort scratch: keys, values, digit counts
    int32_t *s_tv, *s_rh;
    float4 *sym_sorted;      // charges ordered by charge value (negative first)
    int32_t *sym_perm;       // sorted slot -> state index
    int32_t *sym_bcnt;       // per-block counts / offsets of the partition
    float *sym_tileq;        // per tile: the common charge of its slots, NaN if they differ
    int sym_grid, sym_cap;
    // stage timing (obem_profile)
    int prof_on;
    int prof_n;                      // recorded steps (ring of OBEM_PROF_MAX)
    cudaEvent_t *prof_ev;            // [OBEM_PROF_MAX][OBEM_PROF_EV]
    unsigned long long *d_counters;  // [OBEM_NCOUNTERS]: see FieldLaunch::counters
    long long launches;              // kernels launched by recorded steps
    long long steps_recorded;
};
#define OBEM_PROF_MAX 256
#define OBEM_PROF_EV 6   // step start, after cells, after pairs, step end, near start, near end

// ---------------------------------------------------------------- error helpers
int obem_fail(obem_ctx *ctx, int code, const char *fmt, ...);
#define OBEM_CUDA(ctx, call)                                                              \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return obem_fail((ctx), OBEM_ERR_CUDA, "%s failed: %s (%s:%d)", #call,        \
                             cudaGetErrorString(e_), __FILE__, __LINE__);                 \
    } while (0)
#define OBEM_LAUNCH(ctx)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return obem_fail((ctx), OBEM_ERR_CUDA, "kernel launch failed: %s (%s:%d)",    \
                             cudaGetErrorString(e_), __FILE__, __LINE__);                 \
    } while (0)

// ---------------------------------------------------------------- entry points between TUs
// field.cu
struct FieldLaunch {
    const float4 *targets;
    const int32_t *nt_dev;   // device count (step) or NULL
    int nt;
    const float4 *sources;   // NULL: no Coulomb part
    const int32_t *ns_dev;
    int ns;
    int self_exclude;
    int shard;               // the targets are a slice of the sources (a shard's own charges inside the
                             // gathered charges of every shard): one-sided kernel only
    int self_off;            // with self_exclude: target t is source t + self_off (0: targets are the sources)
    float eps2;              // Plummer softening squared (m^2)
    const float *sigma;      // NULL: no cell part
    PanelsDev panels;
    float4 *E_out;
    float3 e_ext;
    int want_v;
    // optional counters [OBEM_NCOUNTERS]: charge pairs; (target block, cell)
    // pairs by tier: 1 point, 3-6 points, 7 or more; (target, cell) pairs in
    // the FP64 closed form; (target, quadrature point) evaluations; (target,
    // cell) pairs evaluated by quadrature
    unsigned long long *counters;
    // optional events: [1] after the cell kernels, [2] after the all-pairs kernel,
    // [4] / [5] around the near-cell kernel
    cudaEvent_t *events;
    // cell kernels: target order (spatially binned) or NULL for the given order,
    // and the block list over that order (NULL: blocks of CT_BLOCK in order)
    const int32_t *perm;
    const int2 *blocks;
    const int32_t *nblocks;
    // E_out already holds a field to add to (e.g. the interpolated map)
    int add_init;
    // > 0: the charges' field by the approximate N-body method on this grid
    int nn_grid;
    // batch of chambers: chamber of every block of the block list, and each
    // chamber's (first cell, cell count) in the concatenated cell arrays
    const int32_t *block_cham;
    const int2 *cham_pan;
};
// A batch of independent chambers in one concatenated charge state, as the
// symmetric all-pairs kernels see it (nb == 0: no batch).  Chamber c holds
// slots [seg_off[c], seg_off[c + 1]) (multiples of OBEM_SEG_ALIGN), its first
// n[c] live; slot_cham[k] is the chamber of slots [k, k + 1) * OBEM_SEG_ALIGN.
#define OBEM_SEG_ALIGN 1024
struct SymBatch {
    int nb;
    const int32_t *seg_off;      // [nb + 1]
    const int32_t *n;            // [nb]
    const int32_t *slot_cham;    // [seg_off[nb] / OBEM_SEG_ALIGN]
    const long long *joff, *ioff;   // [nb] offsets (floats) of the chamber's partial sums
    int32_t *uoff;               // [nb + 1] work units before each chamber (written per launch)
    int32_t *negtot;             // [nb] negative charges per chamber (written per launch)
};
// Far cells in groups (OBEM_STEP_CELL_GROUPS): OBEM_GRP_K cells consecutive
// in the Morton order of their centroids form a group; for a target block
// whose box is at least sqrt(OBEM_GRP_THETA2) group radii from the group's
// centre, the group is replaced by OBEM_GRP_M equivalent point charges on the
// sphere of the group's radius, fitted in FP64 to the group's potential at
// OBEM_GRP_CHECK points on a sphere of OBEM_GRP_RC radii.
#define OBEM_GRP_K 32
#define OBEM_GRP_M 49
#define OBEM_GRP_CHECK 147
#define OBEM_GRP_THETA2 81.0f
#define OBEM_GRP_RC 2.5
struct CellGroups {
    int ng;
    const int32_t *perm;     // [np] cell indices in group order (group g: [g K, g K + K))
    const float4 *cr;        // [ng] centre x, y, z and radius (binary32, radius rounded up)
    const float *h2min;      // [ng] smallest h^2 (longest edge squared) of the group's cells
    const float4 *u;         // [OBEM_GRP_M] unit directions of the equivalent charges
    const float *q;          // [ng * OBEM_GRP_M] equivalent charges (k_C q) for the current sigma
};
// cellgroup.cu
int obem_cell_groups_build(obem_ctx *c, const double *tri, const float4 *g0_h, int np);
void obem_cell_groups_free(obem_ctx *c);
int obem_cell_groups_fit(obem_ctx *c, const float *sigma, cudaStream_t s, CellGroups *G, int *launched);
#define OBEM_BINS_PER_AXIS 64
#define OBEM_NBINS (OBEM_BINS_PER_AXIS * OBEM_BINS_PER_AXIS * OBEM_BINS_PER_AXIS)
#define OBEM_SUPER_SHIFT 6                        // super-bin = 4 x 4 x 4 bins
#define OBEM_NSUPER (OBEM_NBINS >> OBEM_SUPER_SHIFT)
int obem_launch_field(obem_ctx *ctx, const FieldLaunch &L, int capacity_targets, cudaStream_t s);
int obem_launch_step_batch(obem_ctx *c, const obem_state *st, const StepBatch &B, const BtScratch &W,
                           const float4 *E, cudaStream_t s);

// Field of a batch of chambers at every live slot: the cells of the slot's
// chamber plus the other charges of its chamber (symmetric all-pairs kernel on
// the chamber's tiles; one persistent launch for every chamber's work).
struct FieldBatch {
    int nb, slots;               // chambers, slots (seg_off[nb])
    int cut;                     // targets per cell-kernel block, <= 512
    int max_blocks;              // sum over chambers of ceil(capacity / cut)
    int cells, charges;          // cell part, all-pairs part
    float eps2;
    float3 e_ext;
    PanelsDev panels;            // concatenated cells of every chamber
    const float *sigma;
    const int2 *cham_pan;        // [nb] (first cell, cell count)
    int2 *blocks;                // [max_blocks] cell-kernel blocks (scratch)
    int32_t *block_cham, *nblocks;
    SymBatch sym;
    float *jpart, *ipart;
    float4 *sorted;
    int32_t *perm, *bcnt;
    float *tileq;
    int *counter;
    int sym_grid;
};
int obem_launch_field_batch(obem_ctx *ctx, const FieldBatch &F, const float4 *pos_q, float4 *E_out,
                            cudaStream_t s);
size_t obem_sym_sizes(int capacity, size_t *ipart_floats);
int obem_cell_layout(const double *tri, const int32_t *kind, int np, float4 *ca, float4 *g0, float4 *g1,
                     float4 *g2, float4 *nr, float4 *cl);
void obem_cell_geo64(const double *tri, int np, double *geo);
size_t obem_sym_jpart_floats(int capacity);
size_t obem_sym_pass_jpart_floats(int capacity);
size_t obem_sym_pass_ipart_floats(int capacity);
size_t obem_sym_ipart_floats(int capacity);
int obem_sym_grid(int device);
int obem_sym_part_blocks(int capacity);
int obem_binsort_blocks(int capacity);
int obem_point_bins_maxblocks(int n);
size_t obem_point_bins_bytes(int n);
int obem_point_bins(obem_ctx *ctx, const float4 *pts, int n, void *scratch, int32_t **perm, int2 **blocks,
                    int32_t **nblocks, cudaStream_t s);
int obem_sym_tiles(int capacity);

// nn.cu
int obem_launch_nbody_nn(obem_ctx *c, const float4 *pos, const int32_t *n_dev, int n, int G, float eps2,
                         float4 *E_out, float3 e_ext, int add, cudaStream_t s);

// fieldmap.cu
int obem_fieldmap_build_nodes(obem_ctx *ctx, const float *sigma, cudaStream_t s);
int obem_fieldmap_interp(obem_ctx *ctx, const float4 *pts, const int32_t *n_dev, int n, float4 *out, float3 e_ext,
                         cudaStream_t s);

// backward.cu
struct BwArgs {
    const float *targets;
    int nt;
    const float *sources;
    int ns;
    int self_exclude;
    const float *sigma;
    PanelsDev panels;
    const float *dL_dE;
    float *dL_dsigma, *dL_dtargets, *dL_dsources;
};
int obem_launch_backward(obem_ctx *ctx, const BwArgs &A, cudaStream_t s);
size_t obem_influence_scratch_bytes(int ns, int np);
int obem_launch_influence(obem_ctx *ctx, const float4 *src, int ns, const PanelsDev &P, double *S, const double *geo,
                          const int *kind, const double *epsd, float *drhs, void *scratch, int selftest,
                          cudaStream_t s);
int obem_selftest_solve_wait(obem_ctx *c, cudaStream_t s);

// step.cu
int obem_launch_step(obem_ctx *ctx, const obem_state *st, const float4 *E, uint32_t step,
                     obem_step_stats *stats, cudaStream_t s);
int obem_launch_surface_sigma(obem_ctx *ctx, float *sigma_free, cudaStream_t s);
int obem_launch_shard_propose(obem_ctx *c, const obem_state *st, const obem_state *G, uint32_t step,
                              unsigned long long *ionkey, cudaStream_t s);
int obem_launch_shard_count(obem_ctx *c, const obem_state *st, const float4 *E, uint32_t step,
                            const unsigned long long *ionkey, int self_off, obem_step_stats *stats, cudaStream_t s);
int obem_launch_shard_commit(obem_ctx *c, const obem_state *st, const float4 *E, uint32_t step, uint32_t id_base,
                             int commit, obem_step_stats *stats, cudaStream_t s);

// bem.cu
int obem_assemble_and_factor(obem_ctx *ctx, int precision, cudaStream_t s);
int obem_factor_dense(obem_ctx *c, const float *A, int n, int precision, cudaStream_t s);
int obem_solve_dense_rhs(obem_ctx *c, const double *b, double *x, obem_solve_report *rep, cudaStream_t s);

// lu_tc.cu: C[M x N] -= A[M x K] B[K x N] (FP32 row-major blocks) with BF16
// operands on the tensor cores, FP32 accumulation; err: device status word
int obem_tc_gemm_sub(obem_ctx *c, float *C, long long ldc, const float *A, long long lda, const float *B,
                     long long ldb, int M, int N, int K, int *err, cudaStream_t s);
int obem_tc_reserve(obem_ctx *c, size_t a_elems, size_t b_elems);
void obem_tc_free(obem_ctx *c);
int obem_solve_system(obem_ctx *ctx, const double *gv, const float *sigma_free, const float *drhs,
                      float *sigma_out, obem_solve_report *rep, cudaStream_t s);
int obem_solve_adjoint(obem_ctx *ctx, const float *g, double *dL_dgv, float *dL_db, obem_solve_report *rep,
                       cudaStream_t s);
