/*
 * obem.h -- C ABI of the GB300 field + tracking-step engine for the
 * OuroborosBEM method (Quemener & Salvador, arXiv 2110.09214).
 *
 * The library evaluates the electric field at every free charge -- the
 * boundary-element (BEM) cell field plus the all-pairs Coulomb field of the
 * other charges -- and advances the charges by one tracking step
 * (free flight, null-collision Monte Carlo on tabulated cross sections,
 * ionisation with stream compaction, attachment, electron-ion recombination).
 *
 * Conventions for every call:
 *   - SI units: metres, seconds, volts, coulombs; cross sections in m^2 on an
 *     energy grid in eV.
 *   - "device" pointers are CUDA global-memory pointers owned by the caller;
 *     "host" pointers are read before the call returns.  The context owns
 *     the BEM matrix, its factors, the gas tables and its scratch memory.
 *   - Calls taking a stream enqueue work on it and return without waiting,
 *     except obem_bem_assemble and obem_bem_solve, which synchronise that
 *     stream (they are set-up calls).  obem_field_eval and obem_step allocate
 *     nothing and never synchronise.
 *   - The return value is an obem_status; on failure obem_last_error()
 *     describes it.  Errors found on the GPU by obem_step are written to
 *     obem_step_stats.status instead.
 *   - Triangles only: a quadrilateral cell is passed as two triangles.
 */
#ifndef OBEM_H
#define OBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *obem_stream;   /* same handle as cudaStream_t */
typedef struct obem_ctx obem_ctx;          /* opaque */

typedef enum {
    OBEM_OK = 0,
    OBEM_ERR_ARG = -1,            /* invalid argument (null pointer, size, range) */
    OBEM_ERR_CUDA = -2,           /* a CUDA runtime or cuBLAS call failed */
    OBEM_ERR_STATE = -3,          /* call out of order (e.g. solve before assemble) */
    OBEM_ERR_SINGULAR = -4,       /* zero pivot in the LU factorisation */
    OBEM_ERR_NOT_CONVERGED = -5,  /* iterative refinement did not converge */
    OBEM_ERR_CAPACITY = -6,       /* step output exceeds capacity; nothing committed */
    OBEM_ERR_TIMEOUT = -7,        /* a bounded device-side wait ran out */
    OBEM_ERR_TRIALS = -8          /* a charge needed more null-collision trials than trial_cap */
} obem_status;

/* Cross-section process kinds (Sec. 3.3: elastic, inelastic, ionisation,
 * attachment) and how the collision frequency of a process is given. */
enum { OBEM_P_ELASTIC = 0, OBEM_P_EXCITATION = 1, OBEM_P_IONISATION = 2, OBEM_P_ATTACHMENT = 3 };
enum { OBEM_MODE_TABLE = 0, OBEM_MODE_CONST = 1 };

/* Cell kinds (Sec. 2.1): electrode-to-dielectric (Dirichlet rows, Eq. (DBC))
 * and dielectric-to-dielectric (Neumann rows, Eq. (NBC)). */
enum { OBEM_CELL_ELECTRODE = 0, OBEM_CELL_DIELECTRIC = 1 };

/* Species of a charge; the charge value itself is in pos_q[4*i+3]. */
enum { OBEM_ELECTRON = 0, OBEM_CATION = 1, OBEM_ANION = 2 };

/* Arithmetic of the trailing updates of the BEM LU factorisation. */
enum {
    OBEM_LU_FP32 = 0,   /* FP32 on the CUDA cores */
    OBEM_LU_TF32 = 1,   /* TF32 tensor cores, FP32 accumulation */
    OBEM_LU_BF16 = 2,   /* recursive LU, every trailing update a hand-written tcgen05 GEMM:
                           BF16 operands, FP32 accumulation into the FP32 factors */
    OBEM_LU_BF16X9 = 3  /* FP32-accurate BF16x9 emulation on the tensor cores */
};

/* obem_step feature flags */
enum {
    OBEM_STEP_SPACE_CHARGE = 1,   /* add the all-pairs Coulomb field, Eq. (nbody) */
    OBEM_STEP_CELL_FIELD = 2,     /* add the BEM cell field, Eq. (BEM3), with the current sigma */
    OBEM_STEP_FIELD_MAP = 4,      /* take the cell field from the static map (obem_fieldmap_build),
                                     interpolated trilinearly; replaces OBEM_STEP_CELL_FIELD */
    OBEM_STEP_PROB_COLLISION = 8, /* the paper's collision sampling (Sec. 3.3.1): one interaction test
                                     per step, probability 1 - exp(-nu_tot(eps) dt), after the step's
                                     flight; default: exact null-collision trials */
    OBEM_STEP_NBODY_NN = 16,      /* the paper's approximate N-body field (Sec. 3.2.4, "NN"; see
                                     obem_nbody_nn_eval) instead of the exact all-pairs sum, with
                                     obem_config.nn_grid cells per axis */
    OBEM_STEP_SURFACE_HITS = 32,  /* cells absorb the charges whose sub-flight chords cross them and
                                     count their charge (charging-up, Sec. 3.2.3; obem_surface_charge) */
    OBEM_STEP_CELL_GROUPS = 64    /* cell field of obem_step and obem_field_eval (not the batch):
                                     groups of 32 cells (Morton order of the centroids) at >= 9 group
                                     radii from a block of targets enter as 49 equivalent charges
                                     fitted in FP64 to the group's potential (refitted when sigma
                                     changes); set at obem_create, built by obem_mesh_load */
};

enum { OBEM_NN_GMAX = 64 };        /* largest nn_grid */

typedef struct obem_config {
    int32_t capacity;       /* largest number of charges obem_step will hold */
    int32_t trial_cap;      /* max null-collision trials per charge per step, 1..256 */
    int32_t flags;          /* OBEM_STEP_* */
    int32_t nn_grid;        /* cells per axis of the approximate N-body field, 1..64 (0: 16) */
    double dt;              /* tracking step (s) */
    uint64_t seed;          /* Philox4x32-10 key */
    double softening;       /* Plummer length of the N-body field in obem_step (m); 0 = exact */
    double z_lo, z_hi;      /* absorbing electrode planes z = z_lo, z = z_hi (m) */
    double beta;            /* recombination rate coefficient (m^3/s): R_c = (3 beta dt / 4 pi)^(1/3);
                               0: R_c from Eq. (distRecomb); < 0: no recombination */
    double e_ext[3];        /* uniform field added at every charge in obem_step (V/m) */
} obem_config;

typedef struct obem_gas {
    int32_t n_proc;             /* number of processes, 1..32 */
    int32_t n_energy;           /* grid points, 2..4096 */
    const float *energy_eV;     /* host [n_energy], strictly increasing */
    const float *sigma_m2;      /* host [n_proc][n_energy], used for OBEM_MODE_TABLE rows */
    const int32_t *kind;        /* host [n_proc], OBEM_P_* */
    const int32_t *mode;        /* host [n_proc], OBEM_MODE_* */
    const float *threshold_eV;  /* host [n_proc]; sigma = 0 below it; energy loss of excitations */
    const float *nu_const;      /* host [n_proc], collision frequency (1/s) of OBEM_MODE_CONST rows */
    double T;                   /* gas temperature (K) */
    double N;                   /* gas number density (m^-3) */
    double M_amu;               /* gas molecule / ion mass (amu); <= 0: infinite (no recoil, ions fixed) */
    double nu_ion;              /* constant ion collision frequency (1/s) */
} obem_gas;

/* Charge state, structure of arrays in device memory, sorted by id. */
typedef struct obem_state {
    float *pos_q;          /* device [capacity][4]: x, y, z (m), q (C) */
    float *vel;            /* device [capacity][4]: vx, vy, vz (m/s), unused */
    uint32_t *id;          /* device [capacity]: unique, increasing */
    uint32_t *birth;       /* device [capacity]: 0 for initial charges, s+1 if created in step s */
    uint8_t *species;      /* device [capacity]: OBEM_ELECTRON / OBEM_CATION / OBEM_ANION */
    int32_t *n;            /* device scalar: live charges; updated by obem_step */
    uint32_t *next_id;     /* device scalar: next unused id; updated by obem_step */
    int32_t capacity;      /* host: length of the arrays; must not exceed obem_config.capacity */
} obem_state;

/* Per-step observables and status, written to device memory by obem_step
 * (Sec. 4.1: swarm parameters are extracted from the cloud moments). */
typedef struct obem_step_stats {
    int32_t status;             /* OBEM_OK, OBEM_ERR_CAPACITY or OBEM_ERR_TRIALS */
    int32_t n_before, n_after;  /* charges before / after the step */
    int32_t required_capacity;  /* charges the step produced (valid also on OBEM_ERR_CAPACITY) */
    int32_t n_electron, n_cation, n_anion;
    int32_t spawned_pairs, absorbed, attached, recombined_pairs, collisions;
    int64_t trials;             /* collision trials (real + null) */
    double sum_e[3], sum2_e[3]; /* electrons: sum of x,y,z and of x^2,y^2,z^2 (m, m^2) */
    double sum_i[3], sum2_i[3]; /* ions (cations + anions) */
    double sum_energy_e;        /* electrons: total kinetic energy (eV) */
} obem_step_stats;

typedef struct obem_solve_report {
    int32_t iterations;         /* refinement iterations done */
    int32_t status;             /* OBEM_OK or OBEM_ERR_NOT_CONVERGED */
    double backward_error;      /* ||b - A s||_inf / (||A||_inf ||s||_inf + ||b||_inf), FP64 residual */
    double factor_ms;           /* time of the last LU factorisation */
    double solve_ms;            /* time of this solve */
} obem_solve_report;

/* Create a context.  cfg is copied; scratch for cfg->capacity charges is
 * allocated here.  Returns OBEM_ERR_ARG for out-of-range fields. */
int obem_create(obem_ctx **ctx, const obem_config *cfg);
void obem_destroy(obem_ctx *ctx);
/* Text of the last error of this context (static storage, never NULL). */
const char *obem_last_error(const obem_ctx *ctx);

/* Load the gas: cross-section tables and the constants of the collision
 * model (Sec. 3.3, Eq. (leth) grid; ion model of Sec. 3.3).  Host arrays are
 * copied to the device. */
int obem_gas_load(obem_ctx *ctx, const obem_gas *gas);

/* Load the cell mesh (Sec. 2.2).  tri_xyz: host [n_panels][3][3] vertices;
 * the normal (v1-v0)x(v2-v0) points from the eps_minus to the eps_plus side.
 * kind: OBEM_CELL_*; group: electrode group of electrode cells (0..n_groups-1),
 * ignored for dielectric cells; eps_minus / eps_plus: relative permittivities
 * (dielectric cells only).  Invalidates any previous factorisation. */
int obem_mesh_load(obem_ctx *ctx, int32_t n_panels, const double *tri_xyz,
                   const int32_t *kind, const int32_t *group, const double *eps_minus,
                   const double *eps_plus, int32_t n_groups);

/* Assemble the dense matrix of Eq. (matrixBEM) -- Q rows (Eq. (BEMpot)) for
 * electrode cells, W rows (Eq. (BEMfld)) for dielectric cells, collocated at
 * the cell centroids, rows equilibrated -- and factorise it (blocked LU with
 * partial pivoting; trailing updates in the arithmetic `precision`,
 * OBEM_LU_*).  Synchronises `stream`. */
int obem_bem_assemble(obem_ctx *ctx, int32_t precision, obem_stream stream);

/* Solve Eq. (matrixBEM) for sigma with the stored factors and iterative
 * refinement (FP64 residuals) -- Sec. 2.2 keeps the factorisation to re-solve
 * for new voltages or free charges.  group_voltage: host [n_groups];
 * sigma_free: device [n_panels] free density of dielectric cells or NULL
 * (Eq. (charge-up)); drhs: device [n_panels] right-hand-side correction or NULL
 * (the influence terms of Eqs. (BEMpotpart), (BEMfldpart)); sigma_out: device
 * [n_panels].  The solution also becomes the context's current sigma used by
 * obem_step.  rep may be NULL.  Synchronises `stream`. */
int obem_bem_solve(obem_ctx *ctx, const double *group_voltage, const float *sigma_free,
                   const float *drhs, float *sigma_out, obem_solve_report *rep,
                   obem_stream stream);

/* Influence of free charges on the cells (Sec. 3.2.2, Eqs. (potpart),
 * (fldpart)): the right-hand-side correction of Eqs. (BEMpotpart),
 * (BEMfldpart) for obem_bem_solve's drhs, so that the cell charges respond
 * to the space charge (the paper's dynamic option):
 *   electrode cell i:   drhs_i = -Vbar_i,  Vbar_i = k_C sum_p q_p phi_i(y_p) / A_i
 *   dielectric cell i:  drhs_i = -(eps+ - eps-) eps0 Ebar_i . n_i,
 *                       Ebar_i = -k_C sum_p q_p F_i(y_p) / A_i
 * i.e. the charges' potential and field averaged over cell i (phi_i, F_i:
 * potential and field of a unit density on cell i; A_i its area; n_i its
 * normal).  sources: device [ns][4] (x, y, z, q), 16-byte aligned; drhs:
 * device [n_panels].  The cell integrals use the quadrature tiers of the
 * field evaluation and the FP64 closed form within one cell size of a charge.
 * OBEM_ERR_STATE without a mesh; OBEM_ERR_TIMEOUT if a bounded wait for a
 * bulk copy of the charges ran out (drhs is then undefined).  Allocates
 * scratch on the first call and whenever ns exceeds every earlier call's;
 * synchronises `stream` (to read the status of its waits). */
int obem_influence_rhs(obem_ctx *ctx, const float *sources, int32_t ns, float *drhs, obem_stream stream);

/* Adjoint of obem_bem_solve, for gradients through the solve.  Given
 * dL_dsigma = dL/dsigma (device [n_panels]), solves A^T mu = dL/dsigma with
 * the stored factors (transposed triangular solves, iterative refinement
 * with FP64 residuals on the equilibrated matrix); mu = dL/db is the
 * gradient with respect to the right-hand side b of Eq. (matrixBEM): on a
 * dielectric cell it is dL/d sigma_free, on every cell dL/d drhs.
 * dL_dgroup_voltage: host [n_groups] or NULL, receives sum of mu over the
 * electrode cells of each group (dL/dV_k); dL_db: device [n_panels] or
 * NULL.  rep may be NULL.  The paper keeps the factorisation to re-solve for
 * new right-hand sides (Sec. 2.2); the adjoint is the same reuse with the
 * transposed factors.  OBEM_ERR_STATE before obem_bem_assemble.  Allocates
 * scratch and synchronises `stream` (a set-up call, like the solve). */
int obem_bem_solve_adjoint(obem_ctx *ctx, const float *dL_dsigma, double *dL_dgroup_voltage,
                           float *dL_db, obem_solve_report *rep, obem_stream stream);

/* Field and potential at nt points (Eqs. (BEM2), (BEM3), (nbody)):
 *   E(r) = k_C sum_j sigma_j int_Cj (r - r')/|r - r'|^3 dA'
 *        + k_C sum_p q_p (r - r_p)/|r - r_p|^3
 * targets: device [nt][4] (x, y, z, unused); sources: device [ns][4]
 * (x, y, z, q) or NULL (ns ignored); self_exclude: targets and sources are the
 * same array and pair (t, t) is skipped (requires nt == ns); sigma: device
 * [n_panels] cell densities of the loaded mesh, or NULL for no cell field;
 * E_out: device [nt][4] (Ex, Ey, Ez, V).  The Coulomb sum is exact (no
 * softening): a source at the exact position of a target other than its
 * own self pair gives a non-finite result. */
int obem_field_eval(obem_ctx *ctx, const float *targets, int32_t nt, const float *sources,
                    int32_t ns, int32_t self_exclude, const float *sigma, float *E_out,
                    obem_stream stream);

/* Backward (vector-Jacobian product) of obem_field_eval, for training or
 * optimisation through the field.  The paper does not differentiate its
 * field; this is the derivative of Eqs. (BEM2), (BEM3), (nbody) as
 * obem_field_eval evaluates them.  Given dL_dE = dL/d(Ex, Ey, Ez, V) per
 * target (device [nt][4]), with d = x_t - y_p:
 *   dL_dsigma[j]      = k_C sum_t gE_t . int_Cj (x_t - r')/|x_t - r'|^3 dA'
 *                                 + gV_t int_Cj dA'/|x_t - r'|
 *   dL_dtargets[t]    = (dE_t/dx_t)^T gE_t - gV_t E_t      (x, y, z, 0)
 *   dL_dsources[p]    = k_C q_p sum_t [-(I/|d|^3 - 3 d d^T/|d|^5) gE_t
 *                                      + gV_t d/|d|^3]        (x, y, z)
 *                       and k_C sum_t gE_t . d/|d|^3 + gV_t/|d|   (w: dL/dq_p)
 * targets, sources, self_exclude and sigma mean what they mean in
 * obem_field_eval (sigma is needed only for the cell part of dL_dtargets;
 * dL_dsigma needs a loaded mesh but not sigma).  Outputs: device arrays, each
 * may be NULL to skip it: dL_dsigma [n_panels], dL_dtargets [nt][4],
 * dL_dsources [ns][4] (needs sources).  With self_exclude the target-role and
 * source-role gradients of a charge are returned separately (add them for
 * the total).  Pairs at zero distance are skipped.  Cells near a target
 * (closer than 1.5 longest edges for dL_dtargets, 1 for dL_dsigma) use the
 * FP64 closed form and its Jacobian; farther cells use quadrature tiers.
 * Errors: OBEM_ERR_ARG for negative sizes, missing inputs, self_exclude
 * without sources of size nt, dL_dsources without sources, or arrays not
 * 16-byte aligned; OBEM_ERR_STATE for sigma or dL_dsigma without a mesh.
 * Allocates nothing and does not synchronise. */
int obem_field_eval_backward(obem_ctx *ctx, const float *targets, int32_t nt, const float *sources,
                             int32_t ns, int32_t self_exclude, const float *sigma, const float *dL_dE,
                             float *dL_dsigma, float *dL_dtargets, float *dL_dsources,
                             obem_stream stream);

/* Static field map (Sec. 2.4: the field precomputed on a grid and
 * interpolated during tracking, the "static" option of Sec. 3.2): evaluates
 * the cell field and potential of Eqs. (BEM3), (BEM2) with densities sigma
 * (device [n_panels]) at the nodes lo + (i, j, k) * (hi - lo) / (dims - 1),
 * 0 <= i < dims[0] etc. (lo, hi: host [3] metres; dims: host [3], each >= 2),
 * and keeps them in the context (16 bytes per node, padded to multiples of 8
 * per axis; a previous map is replaced).  OBEM_ERR_STATE without a mesh,
 * OBEM_ERR_ARG for bad bounds or dims.  Allocates and synchronises `stream`. */
int obem_fieldmap_build(obem_ctx *ctx, const double *lo, const double *hi, const int32_t *dims,
                        const float *sigma, obem_stream stream);

/* Trilinear interpolation of the map at n points (device [n][4], x y z
 * used) into E_out (device [n][4]: Ex, Ey, Ez, V); points outside the map's
 * box take the value at the nearest point of the box.  OBEM_ERR_STATE without
 * a map.  Allocates nothing, does not synchronise. */
int obem_fieldmap_eval(obem_ctx *ctx, const float *points, int32_t n, float *E_out, obem_stream stream);

/* Charging-up (Sec. 3.2.3, Eq. (charge-up)).  With OBEM_STEP_SURFACE_HITS,
 * obem_step tests the chord of every ballistic sub-flight against the loaded
 * cells (Moller-Trumbore in binary32; the earliest crossing, ties to the
 * lower cell index): a charge crossing a cell is absorbed there and its
 * charge (+-1 e) is added to the cell's count when the step commits.  This
 * call reads the counts: sigma_free (device [n_panels] or NULL) receives the
 * free surface density e * count / area on dielectric cells (0 on electrode
 * cells) to pass to obem_bem_solve; counts (host [n_panels] or NULL) the raw
 * counts; reset != 0 zeroes them afterwards.  OBEM_ERR_STATE without a mesh.
 * Synchronises `stream` when counts is given. */
int obem_surface_charge(obem_ctx *ctx, float *sigma_free, int64_t *counts, int32_t reset, obem_stream stream);

/* Approximate N-body field at n charges (Sec. 3.2.4, the paper's "NN"
 * option): the exact softened Coulomb sum of Eq. (nbody) over the charges in
 * the 27 cells around each charge (itself excluded), and for every other cell
 * its positive and its negative charge, each at its charge-weighted centre.
 * Cells: grid^3 cubes of edge W / grid over the charges' bounding box (W its
 * largest extent); a charge's cell is floor((x - lo) * (grid / W)) per axis in
 * binary32.  pos_q: device [n][4] (x, y, z, q); E_out: device [n][4]
 * (Ex, Ey, Ez, 0).  grid: 1..OBEM_NN_GMAX.  softening: Plummer length (m).
 * Repeatable to binary32 rounding, not bit for bit: the charges of a cell
 * are summed in the order a counting sort with atomics leaves them (the exact
 * all-pairs field is bit-reproducible).  Allocates nothing, does not
 * synchronise. */
int obem_nbody_nn_eval(obem_ctx *ctx, const float *pos_q, int32_t n, int32_t grid, double softening,
                       float *E_out, obem_stream stream);

/* One tracking step of all charges in st (Sec. 3.2 - 3.3):
 *   1. field at the step-start positions: E_in (device [capacity][4]) if not
 *      NULL, else evaluated here (cell field with the current sigma, or from
 *      the static map with OBEM_STEP_FIELD_MAP, and/or the softened all-pairs
 *      field, as cfg.flags say, plus cfg.e_ext);
 *   2. recombination: every electron proposes its nearest cation within R_c
 *      (binary32 squared distance, ties to the lower id; cations created in
 *      the previous step exempt), every cation accepts the proposer with the
 *      smallest (d^2, id), both are removed;
 *   3. flight under the step-start field (Euler stepper, Sec. 3.2.5) with
 *      exact null-collision trials (Philox4x32-10 keyed by seed, counter
 *      (id, step, trial, tag)); ionisation spawns an electron and a cation
 *      at the distance of Eq. (distIoni); attachment turns the electron into
 *      an anion; crossing z_lo / z_hi absorbs the charge;
 *   4. compaction: survivors in order, then spawned charges ordered by
 *      (parent, trial, electron before cation) with ids next_id, next_id+1...
 * The update is all-or-nothing: if the result exceeds st->capacity (or the
 * context capacity), or a charge exceeds trial_cap, nothing is written and
 * stats->status says why.  stats: device pointer. */
int obem_step(obem_ctx *ctx, const obem_state *st, const float *E_in, uint32_t step,
              obem_step_stats *stats, obem_stream stream);

/* Sharded tracking step: the charges partitioned among shards (one GPU each,
 * as the paper's multi-GPU runs of Sec. 2.4 and Sec. 3.2.4 divide the work), a
 * shard evaluating the field at its own charges only.  A shard is its own
 * context and obem_state (sorted by id; initially a contiguous id range).  The
 * exchanges between shards are the caller's (collectives among ranks, or
 * plain copies for shards on one GPU); "gathered" means the live charges of
 * every shard concatenated in shard order, this shard's at [self_off,
 * self_off + n).  One step, for every shard, in this order:
 *   1. obem_shard_field: E_out (device [capacity][4]) = cell field (current
 *      sigma) + softened Coulomb field of the ns gathered charges `sources`
 *      (device [ns][4], x y z q) at the shard's charges, the charge itself
 *      excluded, + e_ext -- the field obem_step would compute (Eqs. (BEM3),
 *      (nbody)), summed in another order (one-sided kernel).
 *   2. obem_shard_propose: every electron of the shard proposes the nearest
 *      cation of `gathered` (an obem_state over the gathered arrays, its n the
 *      gathered count) within R_c, ties to the lower id; ionkey (device int64
 *      [gathered capacity]) receives, per gathered cation, the smallest
 *      (d^2 bits << 32 | electron id) of this shard's proposals, INT64_MAX
 *      when none.  The caller reduces ionkey over all shards with MIN.
 *   3. obem_shard_count: with the reduced keys, the recombination outcome of
 *      the shard's charges (an electron recombines when its cation chose it, a
 *      cation when it chose anyone) and the flight / collision pass;
 *      stats->spawned_pairs, required_capacity and status are final; nothing
 *      is written to st.  The caller gathers every shard's spawned_pairs and
 *      status.
 *   4. obem_shard_commit: if every shard's status is OBEM_OK (commit != 0):
 *      spawned charges get ids from id_base = global next_id + 2 x (spawned
 *      pairs of the shards before this one), the state is written, and the
 *      moments computed; st->next_id is left at id_base + 2 x this shard's
 *      spawned pairs (the caller sets every shard's next_id to the global
 *      next_id + 2 x all spawned pairs).  commit == 0: nothing is written
 *      and a shard without an error of its own reports OBEM_ERR_STATE.
 * The union of the shards' states then equals obem_step's result on the
 * union of the charges given the same field: ids, order within each shard,
 * every decision (Philox draws are keyed by id).  The context's capacity must
 * cover the gathered count (its spatial-hash scratch holds every cation).
 * The static map and the approximate N-body field are not sharded
 * (OBEM_ERR_ARG).  None of the calls allocates or synchronises. */
int obem_shard_field(obem_ctx *ctx, const obem_state *st, const float *sources, int32_t ns, int32_t self_off,
                     float *E_out, obem_stream stream);
int obem_shard_propose(obem_ctx *ctx, const obem_state *st, const obem_state *gathered, uint32_t step,
                       int64_t *ionkey, obem_stream stream);
int obem_shard_count(obem_ctx *ctx, const obem_state *st, const float *E, uint32_t step, const int64_t *ionkey,
                     int32_t self_off, obem_step_stats *stats, obem_stream stream);
int obem_shard_commit(obem_ctx *ctx, const obem_state *st, const float *E, uint32_t step, uint32_t id_base,
                      int32_t commit, obem_step_stats *stats, obem_stream stream);

/* Measured ALU rates of the context's GPU, for the roofline of the FP32-bound/* Measured ALU rates of the context's GPU, for the roofline of the FP32-bound
 * field kernels (not part of the method).  Runs dependent-chain kernels on
 * every SM for a few milliseconds each and writes out[7] (host):
 *   out[0] FP32 TFLOP/s of packed f32x2 FMA chains (2 flops per lane-op),
 *   out[1] FP32 lane-operations per SM per clock (same run),
 *   out[2] rsqrt.approx per SM per clock,
 *   out[3] FP32 lane-operations per SM per clock when every twelve come with
 *          one rsqrt (the one-sided all-pairs kernel's mix),
 *   out[4] the SM clock during the FMA run (MHz),
 *   out[5] the same as out[3] for sixteen lane-operations per rsqrt (the
 *          symmetric all-pairs kernel's mix),
 *   out[6] the same for fourteen (the symmetric kernel on tiles of one charge
 *          value).
 * Allocates scratch and synchronises `stream`. */
int obem_alu_rates(obem_ctx *ctx, double *out, obem_stream stream);

/* The factorisation and refinement of obem_bem_assemble / obem_bem_solve on a
 * caller-given dense system, for tests of the LU on arbitrary matrices (the
 * assembled BEM matrices, row-equilibrated and diagonally large, seldom need
 * row swaps) -- the paper's dense solve of Eq. (matrixBEM), Sec. 2.2, without
 * the assembly.  obem_dense_factor: A device [n][n] FP32 row-major (copied),
 * equilibrated and factorised with partial pivoting in the arithmetic
 * `precision` (OBEM_LU_*).  obem_dense_solve: x = A^-1 b, b and x device FP64
 * [n], iterative refinement with FP64 residuals; rep may be NULL.  Only on a
 * context without a mesh (OBEM_ERR_STATE otherwise, and for a solve before
 * the factorisation); OBEM_ERR_SINGULAR for a zero pivot,
 * OBEM_ERR_NOT_CONVERGED if the refinement stalls.  Both allocate and
 * synchronise `stream`. */
int obem_dense_factor(obem_ctx *ctx, const float *A, int32_t n, int32_t precision, obem_stream stream);
int obem_dense_solve(obem_ctx *ctx, const double *b, double *x, obem_solve_report *rep, obem_stream stream);

/* The trailing update of the BF16 LU factorisation on the tensor cores, as a
 * plain call (a building block of obem_bem_assemble with OBEM_LU_BF16, for
 * tests and measurement; the paper's dense solve, Sec. 2.2, Eq. (matrixBEM)):
 *   C[M][N] -= A[M][K] B[K][N]
 * C, A, B: device FP32 row-major arrays with leading dimensions ldc >= N,
 * lda >= K, ldb >= N (elements).  The operands are rounded to BF16 (round to
 * nearest even) and the products accumulated in FP32 by tcgen05.mma in
 * 256 x 256 tiles.  Uses the context's BF16 scratch (grown here: allocates)
 * and synchronises `stream`.  OBEM_ERR_ARG for bad sizes; OBEM_ERR_TIMEOUT if
 * a bounded wait of the pipeline ran out (C is then undefined). */
int obem_tc_gemm(obem_ctx *ctx, float *C, int64_t ldc, const float *A, int64_t lda, const float *B, int64_t ldb,
                 int32_t M, int32_t N, int32_t K, obem_stream stream);

/* Failure-detection self-test of the bounded device wait that the LU panel
 * factorisation uses between its CTAs (no passage in the paper): two blocks
 * wait, as the panel's CTAs wait for each other's pivot candidates of a
 * column, for two candidate records that no block publishes; each gives
 * up after the wait's limit (2 s on the global timer), records
 * OBEM_ERR_TIMEOUT in a device status word and returns, leaving the context
 * usable.  Returns OBEM_OK when the status read back is OBEM_ERR_TIMEOUT,
 * OBEM_ERR_STATE otherwise.  Allocates a few bytes, synchronises `stream`. */
int obem_selftest_wait_timeout(obem_ctx *ctx, obem_stream stream);

/* Failure-detection self-tests of the library's other bounded device waits
 * (no passage in the paper).  which = 0: the LU panel's candidate wait, as
 * obem_selftest_wait_timeout.  which = 1: the flag wait of the one-launch
 * triangular substitutions of obem_bem_solve: one thread block waits for a
 * block row that no block solves (needs a factored system of at least 256
 * cells).  which = 2: the bulk-copy wait of obem_influence_rhs's far pass:
 * every copy's barrier expects 16 bytes more than the copy brings (needs a
 * mesh; the cells' centroids serve as charges).  Each wait gives up after 2 s,
 * records OBEM_ERR_TIMEOUT in a device status word and the kernel returns,
 * leaving the context usable.  Returns OBEM_OK when that status was read
 * back, OBEM_ERR_STATE when it was not or the preconditions fail,
 * OBEM_ERR_ARG for another `which`.  Synchronises `stream`. */
int obem_selftest_waits(obem_ctx *ctx, int32_t which, obem_stream stream);

/* Stage timing of obem_step, for measurement (not part of the method).
 * obem_profile(ctx, 1) starts recording CUDA events on the step's stream
 * around its stages (up to 256 steps are kept; older ones are dropped) and
 * counting the evaluations below (the cell kernels then run in their counting
 * variants, a few per cent slower); obem_profile(ctx, OBEM_PROFILE_TIMES)
 * records the events only (counts[2..6] stay 0);
 * obem_stage_times() waits for the recorded events and returns, summed over
 * the recorded steps:
 *   ms[0] cell field (binning + near + far kernels), ms[1] all-pairs field
 *   kernel, ms[2] step kernels (recombination, flight, compaction, moments),
 *   ms[3] whole obem_step, ms[4] the near-cell kernel alone (part of ms[0]);
 *   counts[0] steps recorded, counts[1] kernels launched by those steps,
 *   counts[2] charge pairs of the all-pairs kernel,
 *   counts[3..5] (block of targets, cell) pairs of the far-cell kernel by
 *   quadrature tier (centroid, 3 to 6 points, 7 or more points; counts[5]
 *   also counts (block, cell) pairs of the near-cell rules),
 *   counts[6] (target, cell) pairs evaluated in the FP64 closed form,
 *   counts[7] (target, quadrature point) evaluations of the far- and near-cell
 *   kernels (a separated cell group's equivalent charges count as points),
 *   counts[8] (target, cell) pairs evaluated by quadrature.
 * Recording is then reset.  obem_profile(ctx, 0) stops recording. */
#define OBEM_PROFILE_TIMES 2
int obem_profile(obem_ctx *ctx, int32_t enable);
int obem_stage_times(obem_ctx *ctx, double *ms /* [5] */, int64_t *counts /* [9] */);

/* Field evaluation that allocates no memory and needs no context.
 *
 * There is no counterpart in the paper: this entry point exists for callers
 * that cannot call cudaMalloc -- plug-ins held to a host application's fixed
 * device-memory budget, real-time loops that cannot take the latency or the
 * possible failure of an allocation, code whose host framework owns every
 * allocation -- and so cannot create an obem_ctx (obem_create and
 * obem_mesh_load allocate).
 *
 * It computes what obem_field_eval computes (the cell field plus the Coulomb
 * field of the charges) with the same kernels, but all of its scratch memory
 * is one fixed array compiled into the library (about 5 MB, held on every
 * GPU that loads the library until the process exits).  Inputs and outputs
 * are the caller's:
 *   targets   device [nt][4] (x, y, z, unused), nt <= OBEM_NOALLOC_MAX_TARGETS
 *   sources   device [ns][4] (x, y, z, q) or NULL
 *   cell_xyz  device [np][3][3] FP64 cell vertices (layout of obem_mesh_load's
 *             tri_xyz), np <= OBEM_NOALLOC_MAX_CELLS; np == 0: no cell field
 *   sigma     device [np] cell densities
 *   E_out     device [nt][4] (Ex, Ey, Ez, V)
 *   err       optional host buffer of err_len bytes for an error message
 * Sizes beyond the maxima return OBEM_ERR_ARG with a message in err; nothing
 * is launched then.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, and caches it; make
 * that first call before any stream capture begins.  Every call reuses
 * the same array and leaves its contents behind: two calls whose work
 * overlaps on the GPU (on different streams, or from different host threads)
 * race on it and give wrong results; serialise them on one stream. */
enum { OBEM_NOALLOC_MAX_TARGETS = 262144, OBEM_NOALLOC_MAX_CELLS = 16384 };
int obem_field_eval_noalloc(const float *targets, int32_t nt, const float *sources, int32_t ns,
                            int32_t self_exclude, const double *cell_xyz, const float *sigma,
                            int32_t np, float *E_out, char *err, int32_t err_len,
                            obem_stream stream);

/* Batch of independent chambers (many chambers with uneven charge counts
 * stepped together, e.g. a sweep of the parallel-plate counter of Sec. 4.1
 * over gaps and fields).  Each chamber is the method of obem_step on its own:
 * the field at a charge is the cell field of its chamber's cells (Eq. (BEM3))
 * plus the Coulomb field of the other charges of its chamber (Eq. (nbody)),
 * and the tracking step (Secs. 3.2-3.3) draws from its chamber's Philox key
 * and its own id, so a chamber evolves bit for bit as it would alone given
 * the same field.  Every stage is one launch for all chambers.
 *
 * The charges live in one concatenated state (obem_state): chamber c owns
 * slots [seg_off[c], seg_off[c + 1]) of every array, with its capacity
 * rounded up to a multiple of 1024 (it may fill the whole segment), and its
 * live charges are the first n[c] of them; st->n and st->next_id are device
 * arrays of n_chambers entries and st->capacity is seg_off[n_chambers].
 *
 * obem_batch_create: the batch borrows ctx (which must outlive it) for the gas
 *   (obem_gas_load first), dt, softening, beta, trial_cap, e_ext and flags
 *   (only OBEM_STEP_SPACE_CHARGE, OBEM_STEP_CELL_FIELD and
 *   OBEM_STEP_PROB_COLLISION are allowed); per chamber (host arrays
 *   [n_chambers]): capacity >= 1, absorbing planes z_lo < z_hi, Philox key.
 *   Allocates every buffer the steps need.
 * obem_batch_layout: seg_off (host int64 [n_chambers + 1]).
 * obem_batch_cells: chamber's cells (host FP64 [n_cells][3][3], layout of
 *   obem_mesh_load) and their densities (host [n_cells], C/m^2, e.g. from
 *   obem_bem_solve on a context holding that chamber's mesh); copied; the
 *   next field / step uploads them (synchronously: not during stream capture).
 * obem_batch_field_eval: E_out device [slots][4] (Ex, Ey, Ez, 0) at every live
 *   slot; other slots untouched.
 * obem_batch_step: one step of every chamber (field computed unless E_in,
 *   device [slots][4], is given); the step index is the device scalar *step,
 *   advanced by one when the batch commits; stats device [n_chambers].  If any
 *   chamber fails (OBEM_ERR_CAPACITY / OBEM_ERR_TRIALS in its stats), no
 *   chamber commits and the others report OBEM_ERR_STATE.  Allocates nothing.
 * obem_batch_step_graph: the same fused step, captured once into a CUDA graph
 *   (per set of state, step and stats pointers) and replayed on `stream`.
 * obem_batch_autotune: times the field for cell-kernel blocks of 128, 256 and
 *   512 targets on the current charges (best of reps runs each) and keeps the
 *   fastest; out host [4]: chosen size, its time (ms), the time at 512, 0.
 *   The size changes the field by rounding only (the quadrature tier of a cell
 *   is chosen per block).  obem_batch_set_block sets it directly (32..512). */
typedef struct obem_batch obem_batch;
int obem_batch_create(obem_batch **batch, obem_ctx *ctx, int32_t n_chambers, const int32_t *capacity,
                      const double *z_lo, const double *z_hi, const uint64_t *seed);
void obem_batch_destroy(obem_batch *batch);
int obem_batch_layout(const obem_batch *batch, int64_t *seg_off);
int obem_batch_cells(obem_batch *batch, int32_t chamber, int32_t n_cells, const double *tri_xyz,
                     const float *sigma);
int obem_batch_field_eval(obem_batch *batch, const obem_state *st, float *E_out, obem_stream stream);
int obem_batch_step(obem_batch *batch, const obem_state *st, const float *E_in, uint32_t *step,
                    obem_step_stats *stats, obem_stream stream);
int obem_batch_step_graph(obem_batch *batch, const obem_state *st, uint32_t *step, obem_step_stats *stats,
                          obem_stream stream);
int obem_batch_autotune(obem_batch *batch, const obem_state *st, int32_t reps, double *out, obem_stream stream);
int obem_batch_set_block(obem_batch *batch, int32_t cells_per_block);

#ifdef __cplusplus
}
#endif

#endif /* OBEM_H */
