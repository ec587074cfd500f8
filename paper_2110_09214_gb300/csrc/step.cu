// The tracking step (Sec. 3.2 - 3.3): recombination resolve, free flight with
// exact null-collision trials, ionisation spawn, attachment, absorption on the
// electrode planes, and a deterministic two-pass stream compaction.
//
// Built with --fmad=false: every binary32 operation of the step is one IEEE
// rounding, so that, given the same field, the collision processes, spawns,
// and the compacted order are reproducible bit for bit by any IEEE binary32
// implementation of the same operation sequence.
//
// Passes (all stream-ordered, nothing synchronises):
//   init      zero the stats and the control block
//   partners  nearest eligible cation of every electron (spatial hash, ph_*)
//   resolve   each proposing electron atomicMin's (d^2, e) into its cation
//   count     simulate every charge without writing: survivors, spawn counts,
//             per-block totals for the scan
//   scan      one block: block offsets, totals, capacity check (all-or-nothing)
//   write     simulate again (same counters, same draws) and write survivors
//             and spawned charges to their final slots in scratch
//   commit    copy scratch to the caller's arrays, update n and next_id
//   moments   species counts and cloud moments of the new state
// The bt_* kernels at the end run the same passes for a batch of chambers.
#include "obem_internal.cuh"

#define ST_THREADS 256

typedef unsigned long long u64;

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror & Shaw, SC'11: ten rounds of two 32x32->64 multiplies
// with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniform in [0, 1) from the top 24 bits
__device__ __forceinline__ float unif01(uint32_t u)
{
    return (float)(u >> 8) * 5.9604645e-08f;
}

// -ln(U), U = ((u >> 8) + 1) 2^-24 in (0, 1]: U = 2^(e-24) f with f in [1, 2),
// ln f = 2 atanh((f-1)/(f+1)) summed to the 13th power (basic operations only)
__device__ float neg_log_unif(uint32_t u)
{
    uint32_t m = (u >> 8) + 1u;
    int e = 31 - __clz(m);
    float mf = (float)m;
    float f = mf / (float)(1u << e);
    float t = (f - 1.0f) / (f + 1.0f);
    float t2 = t * t;
    float s = 0.07692308f;
    s = s * t2 + 0.09090909f;
    s = s * t2 + 0.11111111f;
    s = s * t2 + 0.14285715f;
    s = s * t2 + 0.2f;
    s = s * t2 + 0.33333334f;
    s = s * t2 + 1.0f;
    float lnf = 2.0f * t * s;
    float a = (float)(24 - e) * 0.6931472f;
    return a - lnf;
}

// sin, cos of a in [0, pi/2) by their Taylor series in a^2 (Horner)
__device__ __forceinline__ void sincos_quadrant(float a, float &sn, float &cs)
{
    float a2 = a * a;
    float ps = -1.6059044e-10f;
    ps = ps * a2 + 2.5052108e-08f;
    ps = ps * a2 - 2.7557319e-06f;
    ps = ps * a2 + 0.0001984127f;
    ps = ps * a2 - 0.008333334f;
    ps = ps * a2 + 0.16666667f;
    ps = ps * a2 - 1.0f;
    sn = -(a * ps);
    float pc = 2.0876756e-09f;
    pc = pc * a2 - 2.755732e-07f;
    pc = pc * a2 + 2.4801588e-05f;
    pc = pc * a2 - 0.0013888889f;
    pc = pc * a2 + 0.041666668f;
    pc = pc * a2 - 0.5f;
    pc = pc * a2 + 1.0f;
    cs = pc;
}

// isotropic unit vector: cos(theta) = 1 - 2u, azimuth 2 pi u' with the
// quadrant taken from the two top bits of u''s 24-bit fraction
__device__ __forceinline__ float3 isotropic(uint32_t ua, uint32_t ub)
{
    float c = 1.0f - 2.0f * unif01(ua);
    float cc = c * c;
    float om = 1.0f - cc;
    if (om < 0.0f) om = 0.0f;
    float s = sqrtf(om);
    uint32_t b = ub >> 8;
    uint32_t q = b >> 22;
    float f = (float)(b & 0x3FFFFFu) * 5.9604645e-08f;
    float a = f * 6.2831855f;
    float sa, ca;
    sincos_quadrant(a, sa, ca);
    float cp, sp;
    if (q == 0u) { cp = ca; sp = sa; }
    else if (q == 1u) { cp = -sa; sp = ca; }
    else if (q == 2u) { cp = -ca; sp = -sa; }
    else { cp = sa; sp = -ca; }
    return make_float3(s * cp, s * sp, c);
}

// next representable float from x toward +inf (dir > 0) or -inf
__device__ __forceinline__ float next_toward(float x, float dir)
{
    if (x == 0.0f) return dir > 0.0f ? __int_as_float(1) : __int_as_float((int)0x80000001u);
    int b = __float_as_int(x);
    bool up = dir > 0.0f;
    bool pos = x > 0.0f;
    return __int_as_float(up == pos ? b + 1 : b - 1);
}

// grid segment and weight of energy eps (linear interpolation in energy)
__device__ __forceinline__ void egrid_locate(const GasDev &g, float eps, int &lo, float &w)
{
    int hi = g.n_e - 1;
    lo = 0;
    if (eps < __ldg(&g.egrid[0])) { lo = 0; w = 0.0f; }
    else if (eps >= __ldg(&g.egrid[g.n_e - 1])) { lo = g.n_e - 2; w = 1.0f; }
    else {
        while (hi - lo > 1) {
            int mid = (lo + hi) / 2;
            if (__ldg(&g.egrid[mid]) <= eps) lo = mid; else hi = mid;
        }
        float e0 = __ldg(&g.egrid[lo]), e1 = __ldg(&g.egrid[lo + 1]);
        w = (eps - e0) / (e1 - e0);
    }
}

// collision frequency of process j (zero below its threshold)
__device__ __forceinline__ float nu_proc(const GasDev &g, int j, float eps, float Ns, int lo, float w)
{
    if (g.mode[j] == OBEM_MODE_CONST) return g.nuc[j];
    const float *row = g.xs + (size_t)j * g.n_e;
    float s0 = __ldg(&row[lo]);
    float s1 = __ldg(&row[lo + 1]);
    float ds = s1 - s0;
    float sg = s0 + w * ds;
    if (eps < g.thr[j]) sg = 0.0f;
    return Ns * sg;
}

// ------------------------------------------------------------------ one charge
__device__ __forceinline__ ChamberP chamber_of(const GasDev &g)
{
    ChamberP c;
    c.seed_lo = g.seed_lo; c.seed_hi = g.seed_hi; c.z_lo = g.z_lo; c.z_hi = g.z_hi;
    return c;
}

struct FlightOut {
    int dead, attached, nsp, collisions, trials, overflow;
    int hit_cell;         // cell that absorbed the charge, or -1
};

// One collision trial at the charge's current state: with x uniform in
// [0, scale), process j is taken when x < nu_1 + ... + nu_j (none: null).
// Returns 0 when nothing happened (null, or ionisation without the energy),
// 1 after a collision, 2 when the flight ends (attachment).
template <bool EMIT>
__device__ int collide(const GasDev &g, const ChamberP &cp, uint32_t id, uint32_t step, uint32_t k, const uint4 &r, float x,
                       float3 &p, float3 &v, uint8_t &sp, FlightOut &fo, float4 *o_pos, float4 *o_vel,
                       uint32_t *o_id, uint32_t *o_birth, uint8_t *o_sp, int sbase, uint32_t id_base)
{
    float v2 = v.x * v.x + v.y * v.y + v.z * v.z;
    float speed = sqrtf(v2);
    if (sp == OBEM_ELECTRON) {
        float eps = g.K_e * v2;
        int lo;
        float w;
        egrid_locate(g, eps, lo, w);
        float Ns = g.N * speed;
        float cum = 0.0f;
        int proc = -1;
        for (int j = 0; j < g.n_proc; ++j) {
            cum = cum + nu_proc(g, j, eps, Ns, lo, w);
            if (x < cum) { proc = j; break; }
        }
        if (proc < 0) return 0;
        const int kind = g.kind[proc];
        if (kind == OBEM_P_ELASTIC) {
            float3 d = isotropic(r.z, r.w);
            float cosx = 0.0f;
            if (speed > 0.0f) cosx = (v.x * d.x + v.y * d.y + v.z * d.z) / speed;
            float om = 1.0f - cosx;
            float loss = g.two_m_over_M * om;
            float f = 1.0f - loss;
            float sn = speed * sqrtf(f);
            v = make_float3(sn * d.x, sn * d.y, sn * d.z);
            fo.collisions += 1;
        } else if (kind == OBEM_P_EXCITATION) {
            float e2 = eps - g.thr[proc];
            if (e2 < 0.0f) e2 = 0.0f;
            float sn = sqrtf(e2 / g.K_e);
            float3 d = isotropic(r.z, r.w);
            v = make_float3(sn * d.x, sn * d.y, sn * d.z);
            fo.collisions += 1;
        } else if (kind == OBEM_P_IONISATION) {
            float er = eps - g.thr[proc];
            er = er - g.E_therm;
            if (!(er > 0.0f)) return 0;
            float half = 0.5f * er;
            float sn = sqrtf(half / g.K_e);
            float3 d = isotropic(r.z, r.w);
            float rr = g.KCE / (2.0f * er);
            float ox = rr * d.x, oy = rr * d.y, oz = rr * d.z;
            float3 pn = make_float3(p.x + ox, p.y + oy, p.z + oz);
            float3 pp = make_float3(p.x - ox, p.y - oy, p.z - oz);
            if (pn.x == p.x && pn.y == p.y && pn.z == p.z) {
                int axi = 0;
                float a0 = fabsf(d.x), a1 = fabsf(d.y), a2 = fabsf(d.z);
                if (a1 > a0) axi = 1;
                if (a2 > (axi == 1 ? a1 : a0)) axi = 2;
                if (axi == 0) { pn.x = next_toward(p.x, d.x); pp.x = next_toward(p.x, -d.x); }
                else if (axi == 1) { pn.y = next_toward(p.y, d.y); pp.y = next_toward(p.y, -d.y); }
                else { pn.z = next_toward(p.z, d.z); pp.z = next_toward(p.z, -d.z); }
            }
            if (EMIT) {
                uint4 r2 = philox4x32_10(make_uint4(id, step, k, 1u), cp.seed_lo, cp.seed_hi);
                float3 di = isotropic(r2.x, r2.y);
                int slot = sbase + 2 * fo.nsp;
                o_pos[slot] = make_float4(pn.x, pn.y, pn.z, -(float)OBEM_QE);
                o_vel[slot] = make_float4(sn * d.x, sn * d.y, sn * d.z, 0.0f);
                o_id[slot] = id_base + (uint32_t)(2 * fo.nsp);
                o_birth[slot] = step + 1u;
                o_sp[slot] = OBEM_ELECTRON;
                o_pos[slot + 1] = make_float4(p.x, p.y, p.z, (float)OBEM_QE);
                o_vel[slot + 1] = make_float4(g.v_th_ion * di.x, g.v_th_ion * di.y, g.v_th_ion * di.z, 0.0f);
                o_id[slot + 1] = id_base + (uint32_t)(2 * fo.nsp + 1);
                o_birth[slot + 1] = step + 1u;
                o_sp[slot + 1] = OBEM_CATION;
            }
            p = pp;
            v = make_float3(-sn * d.x, -sn * d.y, -sn * d.z);
            fo.nsp += 1;
            fo.collisions += 1;
        } else {
            float3 d = isotropic(r.z, r.w);
            v = make_float3(g.v_th_ion * d.x, g.v_th_ion * d.y, g.v_th_ion * d.z);
            sp = OBEM_ANION;
            fo.attached = 1;
            fo.collisions += 1;
            return 2;
        }
    } else {
        float3 d = isotropic(r.z, r.w);
        float sn = (x < g.half_nu_ion) ? speed : g.v_th_ion;
        v = make_float3(sn * d.x, sn * d.y, sn * d.z);
        fo.collisions += 1;
    }
    return 1;
}

// First cell crossed by the segment a -> b (the chord of one sub-flight), by
// the Moller-Trumbore test in binary32 with the oracle's operation order
// (this file is compiled without contraction): edges e1 = v1 - v0,
// e2 = v2 - v0, d = b - a, h = d x e2, det = e1.h (0: no hit), s = a - v0,
// u = (s.h)/det in [0, 1], q = s x e1, v = (d.q)/det >= 0 with u + v <= 1,
// t = (e2.q)/det in [0, 1]; smallest t, ties to the lower cell index.  Only
// the cells listed in the grid cells the segment's bounding box touches are
// tested (every cell is listed in all grid cells its own box touches, plus
// one on every side).  Returns the cell or -1.
__device__ int seg_hit(const GasDev &g, float3 a, float3 b)
{
    int lo[3], hi[3];
    const float mn[3] = {fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z)};
    const float mx[3] = {fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float t0 = (mn[k] - g.hlo[k]) * g.hinv, t1 = (mx[k] - g.hlo[k]) * g.hinv;
        if (!(t1 >= -1.0f) || !(t0 <= (float)g.hdim[k])) return -1;   // outside the grid (or NaN)
        lo[k] = max(0, min(g.hdim[k] - 1, (int)floorf(t0)));
        hi[k] = max(0, min(g.hdim[k] - 1, (int)floorf(t1)));
    }
    const float d0 = b.x - a.x, d1 = b.y - a.y, d2 = b.z - a.z;
    int best = -1;
    float bt = 0.0f;
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                const int q = (z * g.hdim[1] + y) * g.hdim[0] + x;
                for (int m = g.hstart[q]; m < g.hstart[q + 1]; ++m) {
                    const int k = g.htri[m];
                    const float *v = g.tri9 + 9 * (size_t)k;
                    const float e10 = v[3] - v[0], e11 = v[4] - v[1], e12 = v[5] - v[2];
                    const float e20 = v[6] - v[0], e21 = v[7] - v[1], e22 = v[8] - v[2];
                    const float h0 = d1 * e22 - d2 * e21, h1 = d2 * e20 - d0 * e22, h2 = d0 * e21 - d1 * e20;
                    const float det = e10 * h0 + e11 * h1 + e12 * h2;
                    if (det == 0.0f) continue;
                    const float inv = 1.0f / det;
                    const float s0 = a.x - v[0], s1 = a.y - v[1], s2 = a.z - v[2];
                    const float u = (s0 * h0 + s1 * h1 + s2 * h2) * inv;
                    if (!(u >= 0.0f && u <= 1.0f)) continue;
                    const float q0 = s1 * e12 - s2 * e11, q1 = s2 * e10 - s0 * e12, q2 = s0 * e11 - s1 * e10;
                    const float w = (d0 * q0 + d1 * q1 + d2 * q2) * inv;
                    if (!(w >= 0.0f && u + w <= 1.0f)) continue;
                    const float t = (e20 * q0 + e21 * q1 + e22 * q2) * inv;
                    if (!(t >= 0.0f && t <= 1.0f)) continue;
                    if (best < 0 || t < bt || (t == bt && k < best)) { best = k; bt = t; }
                }
            }
    return best;
}

// ballistic flight for time fl under acceleration a (half a in h); returns
// true when the charge crossed an absorbing plane
__device__ __forceinline__ bool flight(const GasDev &g, const ChamberP &cp, float3 &p, float3 &v, float ax, float ay, float az,
                                       float hx, float hy, float hz, float fl)
{
    {
        float w = hx * fl; float xx = v.x + w; float y = xx * fl; p.x = p.x + y; float dv = ax * fl; v.x = v.x + dv;
    }
    {
        float w = hy * fl; float xx = v.y + w; float y = xx * fl; p.y = p.y + y; float dv = ay * fl; v.y = v.y + dv;
    }
    {
        float w = hz * fl; float xx = v.z + w; float y = xx * fl; p.z = p.z + y; float dv = az * fl; v.z = v.z + dv;
    }
    return p.z <= cp.z_lo || p.z >= cp.z_hi;
}

// Flight of charge i over one step under the field E (Euler in the field,
// exact ballistic motion between trials).  Collision sampling: null-collision
// trials at exponential waiting times -ln(U)/nu_max, process j with
// probability nu_j(eps)/nu_max (coll_mode 0); or the paper's per-step scheme
// (coll_mode 1): flight over the whole step, then one interaction when
// -ln(U) < nu_tot(eps) dt, of type j with probability nu_j/nu_tot.
// Ionisation products at the distance of Eq. (distIoni).  A charge is
// absorbed where a sub-flight's chord crosses a cell (g.hit_on: charging-up)
// or where it ends beyond a plane z_lo / z_hi.  When EMIT is set,
// spawned pairs are written to o_* at slots sbase, sbase+1...
template <bool EMIT>
__device__ void fly(const GasDev &g, const ChamberP &cp, uint32_t id, uint32_t step, float3 &p, float3 &v, uint8_t &sp,
                    float3 E, FlightOut &fo, float4 *o_pos, float4 *o_vel, uint32_t *o_id,
                    uint32_t *o_birth, uint8_t *o_sp, int sbase, uint32_t id_base)
{
    const int s = sp;
    const float qm = g.qm[s];
    const float ax = qm * E.x, ay = qm * E.y, az = qm * E.z;
    const float hx = 0.5f * ax, hy = 0.5f * ay, hz = 0.5f * az;
    if (g.coll_mode == 1) {
        const float3 p0 = p;
        const bool crossed = flight(g, cp, p, v, ax, ay, az, hx, hy, hz, g.dt);
        if (g.hit_on && (fo.hit_cell = seg_hit(g, p0, p)) >= 0) { fo.dead = 1; return; }
        if (crossed) { fo.dead = 1; return; }
        const uint4 r = philox4x32_10(make_uint4(id, step, 1u, 0u), cp.seed_lo, cp.seed_hi);
        fo.trials += 1;
        float nu_tot;
        if (s == OBEM_ELECTRON) {
            float v2 = v.x * v.x + v.y * v.y + v.z * v.z;
            float speed = sqrtf(v2);
            float eps = g.K_e * v2;
            int lo;
            float w;
            egrid_locate(g, eps, lo, w);
            float Ns = g.N * speed;
            nu_tot = 0.0f;
            for (int j = 0; j < g.n_proc; ++j) nu_tot = nu_tot + nu_proc(g, j, eps, Ns, lo, w);
        } else {
            nu_tot = g.nu_ion;
        }
        float pr = nu_tot * g.dt;
        if (!(neg_log_unif(r.x) < pr)) return;
        collide<EMIT>(g, cp, id, step, 1u, r, unif01(r.y) * nu_tot, p, v, sp, fo, o_pos, o_vel, o_id, o_birth,
                      o_sp, sbase, id_base);
        return;
    }
    const float numax = (s == OBEM_ELECTRON) ? g.nu_max_e : g.nu_ion;
    float t = 0.0f;
    uint32_t k = 0;
    for (;;) {
        float tau;
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (numax > 0.0f) {
            k += 1u;
            if ((int)k > g.trial_cap) { fo.overflow = 1; return; }
            r = philox4x32_10(make_uint4(id, step, k, 0u), cp.seed_lo, cp.seed_hi);
            tau = neg_log_unif(r.x) / numax;
        } else {
            tau = __int_as_float(0x7f800000);
        }
        float tn = t + tau;
        float fl = (tn >= g.dt) ? (g.dt - t) : tau;
        const float3 p0 = p;
        const bool crossed = flight(g, cp, p, v, ax, ay, az, hx, hy, hz, fl);
        if (g.hit_on && (fo.hit_cell = seg_hit(g, p0, p)) >= 0) { fo.dead = 1; return; }
        if (crossed) { fo.dead = 1; return; }
        if (tn >= g.dt) return;
        t = tn;
        fo.trials += 1;
        if (collide<EMIT>(g, cp, id, step, k, r, unif01(r.y) * numax, p, v, sp, fo, o_pos, o_vel, o_id, o_birth,
                          o_sp, sbase, id_base) == 2)
            return;
    }
}

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ int cur_n(const obem_state &st) { return *st.n; }

__global__ void init_kernel(obem_step_stats *stats, StepCtl *ctl, const obem_state st)
{
    if (threadIdx.x == 0) {
        memset(stats, 0, sizeof(obem_step_stats));
        memset(ctl, 0, sizeof(StepCtl));
        stats->n_before = *st.n;
    }
}

// ---------------------------------------------------------------- partner search
// Nearest eligible cation within R_c for every electron, by spatial hashing:
// cells of edge h = R_c (1 + 1e-5) are hashed into PH_BUCKETS buckets, the
// eligible cations (not created in the previous step) are counting-sorted by
// bucket, and each electron scans the buckets of its 27 neighbouring cells,
// keeping the smallest (binary32 d^2, index) key with d^2 <= R_c^2.  Every
// cation within R_c lies in one of those cells and hash collisions only add
// candidates that the distance test rejects, so the result is the exact
// minimum over all cations (the same key as a brute-force scan, whatever the
// order in a bucket).  Cell coordinates are computed in FP64 (exact floor to
// ~1e-8 of a cell at metre-scale positions).
#define PH_BUCKETS (1 << 20)

__device__ __forceinline__ uint32_t ph_hash(long long cx, long long cy, long long cz)
{
    const uint32_t h = ((uint32_t)cx * 73856093u) ^ ((uint32_t)cy * 19349663u) ^ ((uint32_t)cz * 83492791u);
    return h & (PH_BUCKETS - 1);
}

__device__ __forceinline__ long long ph_coord(float x, double inv_h)
{
    const double c = floor((double)x * inv_h);
    return (long long)fmin(fmax(c, -4.0e18), 4.0e18);   // in range for the conversion
}
__device__ __forceinline__ void ph_cell(float4 p, double inv_h, long long &cx, long long &cy, long long &cz)
{
    cx = ph_coord(p.x, inv_h);
    cy = ph_coord(p.y, inv_h);
    cz = ph_coord(p.z, inv_h);
}

__global__ void ph_count_kernel(const obem_state st, uint32_t step, double inv_h, int32_t *bucket_of,
                                int32_t *count)
{
    const int n = cur_n(st);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = st.birth[i];
    if (st.species[i] != OBEM_CATION || (b != 0u && b == step)) { bucket_of[i] = -1; return; }
    long long cx, cy, cz;
    ph_cell(reinterpret_cast<const float4 *>(st.pos_q)[i], inv_h, cx, cy, cz);
    const uint32_t h = ph_hash(cx, cy, cz);
    bucket_of[i] = (int32_t)h;
    atomicAdd(&count[h], 1);
}

// start = exclusive scan of count (PH_BUCKETS + 1 entries), cursor = start, in
// three passes: sums of 1024-bucket blocks, scan of the block sums, scan
// within each block plus its offset.
#define PH_BLK 1024
#define PH_NBLK (PH_BUCKETS / PH_BLK)

// inclusive scan of one value per thread over a 1024-thread block
__device__ __forceinline__ int32_t ph_block_scan(int32_t v, int32_t *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int32_t w = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    return v + (warp > 0 ? s_warp[warp - 1] : 0);
}

__global__ void __launch_bounds__(PH_BLK) ph_blocksum_kernel(const int32_t *count, int32_t *bsum)
{
    __shared__ int32_t s_warp[32];
    const int32_t v = ph_block_scan(count[blockIdx.x * PH_BLK + threadIdx.x], s_warp);
    if (threadIdx.x == PH_BLK - 1) bsum[blockIdx.x] = v;
}

__global__ void __launch_bounds__(PH_BLK) ph_scan_sums_kernel(int32_t *bsum)
{
    __shared__ int32_t s_warp[32];
    const int32_t v = bsum[threadIdx.x];
    const int32_t inc = ph_block_scan(v, s_warp);
    __syncthreads();
    bsum[threadIdx.x] = inc - v;                 // exclusive offsets
    if (threadIdx.x == PH_BLK - 1) bsum[PH_NBLK] = inc;
}

__global__ void __launch_bounds__(PH_BLK) ph_scan_apply_kernel(const int32_t *count, const int32_t *bsum,
                                                                  int32_t *start, int32_t *cursor)
{
    __shared__ int32_t s_warp[32];
    const int i = blockIdx.x * PH_BLK + threadIdx.x;
    const int32_t v = count[i];
    const int32_t ex = ph_block_scan(v, s_warp) - v + bsum[blockIdx.x];
    start[i] = ex;
    cursor[i] = ex;
    if (i == PH_BUCKETS - 1) start[PH_BUCKETS] = bsum[PH_NBLK];
}

__global__ void ph_scatter_kernel(const obem_state st, const int32_t *bucket_of, int32_t *cursor, int32_t *sorted)
{
    const int n = cur_n(st);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t h = bucket_of[i];
    if (h < 0) return;
    sorted[atomicAdd(&cursor[h], 1)] = i;
}

__global__ void ph_query_kernel(const obem_state st, GasDev g, double inv_h, const int32_t *start,
                                const int32_t *sorted, u64 *prop)
{
    const int n = cur_n(st);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u64 best = ~0ull;
    if (st.species[i] == OBEM_ELECTRON) {
        const float4 pe = reinterpret_cast<const float4 *>(st.pos_q)[i];
        long long cx, cy, cz;
        ph_cell(pe, inv_h, cx, cy, cz);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const uint32_t h = ph_hash(cx + dx, cy + dy, cz + dz);
                    for (int k = start[h]; k < start[h + 1]; ++k) {
                        const int c = sorted[k];
                        const float4 pc = reinterpret_cast<const float4 *>(st.pos_q)[c];
                        const float ex = pe.x - pc.x, ey = pe.y - pc.y, ez = pe.z - pc.z;
                        const float d2 = ex * ex + ey * ey + ez * ez;
                        if (!(d2 <= g.rc2)) continue;
                        const u64 key = ((u64)__float_as_uint(d2) << 32) | (u64)(uint32_t)c;
                        if (key < best) best = key;
                    }
                }
    }
    prop[i] = best;
}

__global__ void resolve_kernel(const obem_state st, const u64 *prop, u64 *ionkey)
{
    const int n = cur_n(st);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u64 pr = prop[i];
    if (pr == ~0ull || st.species[i] != OBEM_ELECTRON) return;
    uint32_t ion = (uint32_t)(pr & 0xFFFFFFFFu);
    u64 key = (pr & 0xFFFFFFFF00000000ull) | (u64)(uint32_t)i;
    atomicMin(&ionkey[ion], key);
}

__device__ __forceinline__ bool recombined(int i, uint8_t s, const u64 *prop, const u64 *ionkey, int recomb_on)
{
    if (!recomb_on) return false;
    if (s == OBEM_CATION) return ionkey[i] != ~0ull;
    if (s == OBEM_ELECTRON) {
        u64 pr = prop[i];
        if (pr == ~0ull) return false;
        uint32_t ion = (uint32_t)(pr & 0xFFFFFFFFu);
        return ionkey[ion] == ((pr & 0xFFFFFFFF00000000ull) | (u64)(uint32_t)i);
    }
    return false;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(ST_THREADS)
count_kernel(const obem_state st, GasDev g, const float4 *E, uint32_t step, const u64 *prop,
             const u64 *ionkey, int32_t *keep, int32_t *nsp, int32_t *blk, obem_step_stats *stats,
             StepCtl *ctl, int32_t *s_hit)
{
    __shared__ long long sh[ST_THREADS / 32];
    const int n = cur_n(st);
    int i = blockIdx.x * ST_THREADS + threadIdx.x;
    int kp = 0, ns = 0, absorbed = 0, attached = 0, coll = 0, rec = 0, ovf = 0;
    int hit = -1;
    long long trials = 0;
    if (i < n) {
        uint8_t s = st.species[i];
        if (recombined(i, s, prop, ionkey, g.recomb_on)) {
            rec = (s == OBEM_CATION);
        } else {
            float4 pq = reinterpret_cast<const float4 *>(st.pos_q)[i];
            float4 vv = reinterpret_cast<const float4 *>(st.vel)[i];
            float4 e = E[i];
            float3 p = make_float3(pq.x, pq.y, pq.z), v = make_float3(vv.x, vv.y, vv.z);
            FlightOut fo = {0, 0, 0, 0, 0, 0, -1};
            fly<false>(g, chamber_of(g), st.id[i], step, p, v, s, make_float3(e.x, e.y, e.z), fo, NULL, NULL, NULL,
                       NULL, NULL, 0, 0u);
            if (g.hit_on) hit = fo.hit_cell >= 0 ? (fo.hit_cell << 1) | (pq.w > 0.0f ? 1 : 0) : -1;
            kp = !fo.dead;
            ns = fo.nsp;
            absorbed = fo.dead;
            attached = fo.attached;
            coll = fo.collisions;
            trials = fo.trials;
            ovf = fo.overflow;
        }
        keep[i] = kp;
        nsp[i] = ns;
        if (g.hit_on) s_hit[i] = hit;
    }
    long long t;
    t = block_sum<long long>(kp, sh);
    if (threadIdx.x == 0) blk[2 * blockIdx.x] = (int32_t)t;
    t = block_sum<long long>(ns, sh);
    if (threadIdx.x == 0) blk[2 * blockIdx.x + 1] = (int32_t)t;
    t = block_sum<long long>(absorbed, sh);
    if (threadIdx.x == 0 && t) atomicAdd(&stats->absorbed, (int)t);
    t = block_sum<long long>(attached, sh);
    if (threadIdx.x == 0 && t) atomicAdd(&stats->attached, (int)t);
    t = block_sum<long long>(coll, sh);
    if (threadIdx.x == 0 && t) atomicAdd(&stats->collisions, (int)t);
    t = block_sum<long long>(rec, sh);
    if (threadIdx.x == 0 && t) atomicAdd(&stats->recombined_pairs, (int)t);
    t = block_sum<long long>(trials, sh);
    if (threadIdx.x == 0 && t) atomicAdd((unsigned long long *)&stats->trials, (unsigned long long)t);
    t = block_sum<long long>(ovf, sh);
    if (threadIdx.x == 0 && t) atomicOr(&ctl->trial_overflow, 1);
}

// single block: exclusive scan of the per-block (keep, spawn) totals
__global__ void scan_kernel(const obem_state st, int32_t *blk, obem_step_stats *stats, StepCtl *ctl,
                            int cap)
{
    __shared__ int32_t sk[1024], ss[1024];
    __shared__ int32_t carry_k, carry_s;
    const int n = cur_n(st);
    const int nb = (n + ST_THREADS - 1) / ST_THREADS;
    if (threadIdx.x == 0) { carry_k = 0; carry_s = 0; }
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        int b = c0 + threadIdx.x;
        int vk = b < nb ? blk[2 * b] : 0;
        int vs = b < nb ? blk[2 * b + 1] : 0;
        sk[threadIdx.x] = vk;
        ss[threadIdx.x] = vs;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int ak = threadIdx.x >= off ? sk[threadIdx.x - off] : 0;
            int as = threadIdx.x >= off ? ss[threadIdx.x - off] : 0;
            __syncthreads();
            sk[threadIdx.x] += ak;
            ss[threadIdx.x] += as;
            __syncthreads();
        }
        if (b < nb) {
            blk[2 * b] = carry_k + sk[threadIdx.x] - vk;      // exclusive
            blk[2 * b + 1] = carry_s + ss[threadIdx.x] - vs;
        }
        __syncthreads();
        if (threadIdx.x == 1023) { carry_k += sk[1023]; carry_s += ss[1023]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int nk = carry_k, nsp = carry_s;
        long long total = (long long)nk + 2ll * nsp;
        ctl->n_keep = nk;
        ctl->n_spawn = nsp;
        stats->spawned_pairs = nsp;
        stats->required_capacity = total > 0x7fffffff ? 0x7fffffff : (int)total;
        if (ctl->trial_overflow) {
            ctl->abort = 1;
            stats->status = OBEM_ERR_TRIALS;
        } else if (total > cap) {
            ctl->abort = 1;
            stats->status = OBEM_ERR_CAPACITY;
        }
        stats->n_after = ctl->abort ? n : (int)total;
    }
}

__global__ void __launch_bounds__(ST_THREADS)
write_kernel(const obem_state st, GasDev g, const float4 *E, uint32_t step, const u64 *prop,
             const u64 *ionkey, const int32_t *keep, const int32_t *nsp, const int32_t *blk,
             const StepCtl *ctl, float4 *o_pos, float4 *o_vel, uint32_t *o_id, uint32_t *o_birth,
             uint8_t *o_sp)
{
    __shared__ int32_t wk[ST_THREADS / 32], ws[ST_THREADS / 32];
    if (ctl->abort) return;
    const int n = cur_n(st);
    int i = blockIdx.x * ST_THREADS + threadIdx.x;
    int kp = 0, ns = 0;
    if (i < n) { kp = keep[i]; ns = nsp[i]; }
    // block-local exclusive scan
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ik = kp, is = ns;
    for (int o = 1; o < 32; o <<= 1) {
        int a = __shfl_up_sync(0xffffffffu, ik, o);
        int b = __shfl_up_sync(0xffffffffu, is, o);
        if (lane >= o) { ik += a; is += b; }
    }
    if (lane == 31) { wk[warp] = ik; ws[warp] = is; }
    __syncthreads();
    int pk_ = 0, ps_ = 0;
    for (int w = 0; w < warp; ++w) { pk_ += wk[w]; ps_ += ws[w]; }
    const int out_keep = blk[2 * blockIdx.x] + pk_ + ik - kp;
    const int out_spawn = blk[2 * blockIdx.x + 1] + ps_ + is - ns;
    if (i >= n || (!kp && !ns)) return;
    uint8_t s = st.species[i];
    float4 pq = reinterpret_cast<const float4 *>(st.pos_q)[i];
    float4 vv = reinterpret_cast<const float4 *>(st.vel)[i];
    float4 e = E[i];
    float3 p = make_float3(pq.x, pq.y, pq.z), v = make_float3(vv.x, vv.y, vv.z);
    FlightOut fo = {0, 0, 0, 0, 0, 0, -1};
    const int sbase = ctl->n_keep + 2 * out_spawn;
    const uint32_t id_base = *st.next_id + (uint32_t)(2 * out_spawn);
    fly<true>(g, chamber_of(g), st.id[i], step, p, v, s, make_float3(e.x, e.y, e.z), fo, o_pos, o_vel, o_id, o_birth,
              o_sp, sbase, id_base);
    if (kp) {
        o_pos[out_keep] = make_float4(p.x, p.y, p.z, pq.w);
        o_vel[out_keep] = make_float4(v.x, v.y, v.z, vv.w);
        o_id[out_keep] = st.id[i];
        o_birth[out_keep] = st.birth[i];
        o_sp[out_keep] = s;
    }
}

__global__ void commit_kernel(const obem_state st, const StepCtl *ctl, const float4 *o_pos,
                              const float4 *o_vel, const uint32_t *o_id, const uint32_t *o_birth,
                              const uint8_t *o_sp)
{
    if (ctl->abort) return;
    const int m = ctl->n_keep + 2 * ctl->n_spawn;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        reinterpret_cast<float4 *>(st.pos_q)[i] = o_pos[i];
        reinterpret_cast<float4 *>(st.vel)[i] = o_vel[i];
        st.id[i] = o_id[i];
        st.birth[i] = o_birth[i];
        st.species[i] = o_sp[i];
    }
}

__global__ void finish_kernel(const obem_state st, const StepCtl *ctl)
{
    if (threadIdx.x != 0 || ctl->abort) return;
    *st.n = ctl->n_keep + 2 * ctl->n_spawn;
    *st.next_id = *st.next_id + (uint32_t)(2 * ctl->n_spawn);
}

// charges absorbed by cells this step: deposits[cell] += +-1 (units of e),
// only when the step commits (run before the count of charges is updated)
__global__ void deposit_kernel(const obem_state st, const StepCtl *ctl, const int32_t *s_hit,
                               unsigned long long *deposit)
{
    if (ctl->abort) return;
    const int n = cur_n(st);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t h = s_hit[i];
    if (h >= 0) atomicAdd(&deposit[h >> 1], (h & 1) ? 1ull : ~0ull);   // +1 or -1 (two's complement)
}

// free surface density of Eq. (charge-up): e * deposits / area on dielectric
// cells, 0 on electrode cells
__global__ void surface_sigma_kernel(const long long *deposit, const double *area, const int *kind, int np,
                                     float *sigma_free)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    sigma_free[i] = kind[i] == OBEM_CELL_DIELECTRIC ? (float)(OBEM_QE * (double)deposit[i] / area[i]) : 0.0f;
}

int obem_launch_surface_sigma(obem_ctx *c, float *sigma_free, cudaStream_t s)
{
    surface_sigma_kernel<<<(c->np + 255) / 256, 256, 0, s>>>(c->d_deposit, c->d_area, c->d_kind, c->np, sigma_free);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}

// Cloud moments of the new state.  Counts go to the stats by integer atomics
// (exact in any order); the FP64 sums are reduced per block and the blocks'
// partial sums added by moments_fold_kernel in block order, so the moments
// are the same on every run.
#define NMOM 13    // sum_e[3], sum2_e[3], sum_i[3], sum2_i[3], sum_energy_e

__device__ void moments_block(const obem_state &st, int i, bool live, obem_step_stats *stats, double *part)
{
    __shared__ double shd[ST_THREADS / 32];
    __shared__ long long shl[ST_THREADS / 32];
    int ne = 0, nc = 0, na = 0;
    double v[NMOM];
#pragma unroll
    for (int f = 0; f < NMOM; ++f) v[f] = 0.0;
    if (live) {
        const uint8_t s = st.species[i];
        const float4 p = reinterpret_cast<const float4 *>(st.pos_q)[i];
        const double x[3] = {p.x, p.y, p.z};
        if (s == OBEM_ELECTRON) {
            ne = 1;
            for (int c = 0; c < 3; ++c) { v[c] = x[c]; v[3 + c] = x[c] * x[c]; }
            const float4 u = reinterpret_cast<const float4 *>(st.vel)[i];
            const double v2 = (double)u.x * u.x + (double)u.y * u.y + (double)u.z * u.z;
            v[12] = 0.5 * OBEM_ME * v2 / OBEM_QE;
        } else {
            if (s == OBEM_CATION) nc = 1; else na = 1;
            for (int c = 0; c < 3; ++c) { v[6 + c] = x[c]; v[9 + c] = x[c] * x[c]; }
        }
    }
    long long t;
    t = block_sum<long long>(ne, shl); if (threadIdx.x == 0 && t) atomicAdd(&stats->n_electron, (int)t);
    t = block_sum<long long>(nc, shl); if (threadIdx.x == 0 && t) atomicAdd(&stats->n_cation, (int)t);
    t = block_sum<long long>(na, shl); if (threadIdx.x == 0 && t) atomicAdd(&stats->n_anion, (int)t);
    for (int f = 0; f < NMOM; ++f) {
        const double d = block_sum<double>(v[f], shd);
        if (threadIdx.x == 0) part[f] = d;
    }
}

__global__ void __launch_bounds__(ST_THREADS)
moments_kernel(const obem_state st, obem_step_stats *stats, double *part)
{
    const int n = cur_n(st);
    const int i = blockIdx.x * ST_THREADS + threadIdx.x;
    if (blockIdx.x * ST_THREADS >= n) return;            // a block with no charge adds nothing
    moments_block(st, i, i < n, stats, part + (size_t)NMOM * blockIdx.x);
}

// sum of the nb blocks' partial sums from part (NMOM per block), in block
// order within each thread's stride and a fixed tree across threads (1024)
__device__ void moments_fold(const double *part, int nb, obem_step_stats *stats)
{
    __shared__ double red[1024];
    double *dst[NMOM] = {&stats->sum_e[0], &stats->sum_e[1], &stats->sum_e[2], &stats->sum2_e[0],
                         &stats->sum2_e[1], &stats->sum2_e[2], &stats->sum_i[0], &stats->sum_i[1],
                         &stats->sum_i[2], &stats->sum2_i[0], &stats->sum2_i[1], &stats->sum2_i[2],
                         &stats->sum_energy_e};
    for (int f = 0; f < NMOM; ++f) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(size_t)NMOM * b + f];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) *dst[f] = red[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) moments_fold_kernel(const obem_state st, const double *part,
                                                            obem_step_stats *stats)
{
    const int n = cur_n(st);
    moments_fold(part, (n + ST_THREADS - 1) / ST_THREADS, stats);
}

// ====================================================================
// Sharded step (the charges partitioned among shards, Sec. 2.4 / 3.2.4 run on
// several GPUs): a shard holds its own charges, sorted by id, and sees the
// charges of every shard through gathered copies (G, in shard order; its own
// at [self_off, self_off + n)).  Recombination keys are exchanged as int64 with
// INT64_MAX for "none", so that a signed MIN reduction across shards is the
// unsigned minimum of the keys (valid keys are below 2^63: a finite non-negative
// binary32 d^2 in the high word).
#define SH_NONE 0x7FFFFFFFFFFFFFFFull

// each local electron's nearest cation of the gathered set within R_c: ties to
// the lower cation id (as in the unsharded step, whose array order is id
// order); prop[i] = d^2 bits << 32 | gathered index of that cation
__global__ void sh_query_kernel(const obem_state st, const obem_state G, GasDev g, double inv_h,
                                const int32_t *start, const int32_t *sorted, u64 *prop)
{
    const int n = cur_n(st);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u64 best = ~0ull, best_idx = 0;
    if (st.species[i] == OBEM_ELECTRON) {
        const float4 pe = reinterpret_cast<const float4 *>(st.pos_q)[i];
        long long cx, cy, cz;
        ph_cell(pe, inv_h, cx, cy, cz);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const uint32_t h = ph_hash(cx + dx, cy + dy, cz + dz);
                    for (int k = start[h]; k < start[h + 1]; ++k) {
                        const int c = sorted[k];
                        const float4 pc = reinterpret_cast<const float4 *>(G.pos_q)[c];
                        const float ex = pe.x - pc.x, ey = pe.y - pc.y, ez = pe.z - pc.z;
                        const float d2 = ex * ex + ey * ey + ez * ez;
                        if (!(d2 <= g.rc2)) continue;
                        const u64 key = ((u64)__float_as_uint(d2) << 32) | (u64)G.id[c];
                        if (key < best) { best = key; best_idx = (u64)(uint32_t)c; }
                    }
                }
    }
    prop[i] = best == ~0ull ? ~0ull : ((best & 0xFFFFFFFF00000000ull) | best_idx);
}

// the local electrons' proposals into the gathered cations' keys: (d^2, id)
__global__ void sh_propose_kernel(const obem_state st, const u64 *prop, unsigned long long *ionkey)
{
    const int n = cur_n(st);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u64 pr = prop[i];
    if (pr == ~0ull || st.species[i] != OBEM_ELECTRON) return;
    atomicMin(&ionkey[(uint32_t)(pr & 0xFFFFFFFFu)], (pr & 0xFFFFFFFF00000000ull) | (u64)st.id[i]);
}

__global__ void sh_fill_kernel(unsigned long long *k, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        k[i] = SH_NONE;
}

// the reduced keys as the local arrays of the unsharded step: a local
// electron that won its cation gets prop = ionkey = (d^2, own index) at its
// own index; a local cation that accepted a proposal a key != ~0
__global__ void sh_localize_kernel(const obem_state st, const unsigned long long *ionkey, int self_off, u64 *prop,
                                   u64 *ionloc)
{
    const int n = cur_n(st);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint8_t sp = st.species[i];
    u64 p = ~0ull, k = ~0ull;
    if (sp == OBEM_ELECTRON) {
        const u64 pr = prop[i];
        if (pr != ~0ull &&
            ionkey[(uint32_t)(pr & 0xFFFFFFFFu)] == ((pr & 0xFFFFFFFF00000000ull) | (u64)st.id[i])) {
            p = (pr & 0xFFFFFFFF00000000ull) | (u64)(uint32_t)i;
            k = p;
        }
    } else if (sp == OBEM_CATION) {
        if (ionkey[self_off + i] != SH_NONE) k = 0ull;
    }
    prop[i] = p;
    ionloc[i] = k;
}

static GasDev step_gas(obem_ctx *c)
{
    GasDev g = c->gas;
    g.hit_on = (c->cfg.flags & OBEM_STEP_SURFACE_HITS) && c->np > 0 && c->d_tri9;
    if (g.hit_on) {
        g.tri9 = c->d_tri9;
        g.hstart = c->d_hstart;
        g.htri = c->d_htri;
        for (int k = 0; k < 3; ++k) { g.hlo[k] = c->h_hlo[k]; g.hdim[k] = c->h_hdim[k]; }
        g.hinv = c->h_hinv;
    }
    return g;
}

int obem_launch_shard_propose(obem_ctx *c, const obem_state *stp, const obem_state *Gp, uint32_t step,
                              unsigned long long *ionkey, cudaStream_t s)
{
    const obem_state st = *stp, G = *Gp;
    const int nblk = (st.capacity + ST_THREADS - 1) / ST_THREADS;
    const int gblk = (G.capacity + ST_THREADS - 1) / ST_THREADS;
    const GasDev g = step_gas(c);
    sh_fill_kernel<<<(G.capacity + 255) / 256 < 4096 ? (G.capacity + 255) / 256 : 4096, 256, 0, s>>>(ionkey,
                                                                                                  G.capacity);
    OBEM_LAUNCH(c);
    if (!g.recomb_on || !(g.rc2 > 0.f)) {
        OBEM_CUDA(c, cudaMemsetAsync(c->s_prop, 0xFF, sizeof(u64) * (size_t)st.capacity, s));
        return OBEM_OK;
    }
    // spatial hash of the gathered cations, queried by the local electrons
    const double inv_h = 1.0 / (sqrt((double)g.rc2) * (1.0 + 1e-5));
    OBEM_CUDA(c, cudaMemsetAsync(c->ph_count, 0, sizeof(int32_t) * PH_BUCKETS, s));
    ph_count_kernel<<<gblk, ST_THREADS, 0, s>>>(G, step, inv_h, c->ph_bucket, c->ph_count);
    ph_blocksum_kernel<<<PH_NBLK, PH_BLK, 0, s>>>(c->ph_count, c->ph_bsum);
    ph_scan_sums_kernel<<<1, PH_BLK, 0, s>>>(c->ph_bsum);
    ph_scan_apply_kernel<<<PH_NBLK, PH_BLK, 0, s>>>(c->ph_count, c->ph_bsum, c->ph_start, c->ph_cursor);
    ph_scatter_kernel<<<gblk, ST_THREADS, 0, s>>>(G, c->ph_bucket, c->ph_cursor, c->ph_sorted);
    sh_query_kernel<<<nblk, ST_THREADS, 0, s>>>(st, G, g, inv_h, c->ph_start, c->ph_sorted, c->s_prop);
    sh_propose_kernel<<<nblk, ST_THREADS, 0, s>>>(st, c->s_prop, ionkey);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}

int obem_launch_shard_count(obem_ctx *c, const obem_state *stp, const float4 *E, uint32_t step,
                            const unsigned long long *ionkey, int self_off, obem_step_stats *stats, cudaStream_t s)
{
    const obem_state st = *stp;
    const int cap = st.capacity;
    const int nblk = (cap + ST_THREADS - 1) / ST_THREADS;
    const GasDev g = step_gas(c);
    init_kernel<<<1, 32, 0, s>>>(stats, c->s_ctl, st);
    OBEM_LAUNCH(c);
    if (g.recomb_on) {
        sh_localize_kernel<<<nblk, ST_THREADS, 0, s>>>(st, ionkey, self_off, c->s_prop, c->s_ionkey);
        OBEM_LAUNCH(c);
    }
    count_kernel<<<nblk, ST_THREADS, 0, s>>>(st, g, E, step, c->s_prop, c->s_ionkey, c->s_keep,
                                             c->s_nsp, c->s_blk, stats, c->s_ctl, c->s_hit);
    OBEM_LAUNCH(c);
    scan_kernel<<<1, 1024, 0, s>>>(st, c->s_blk, stats, c->s_ctl, cap < c->cap ? cap : c->cap);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}

// the shard does not commit (another shard's step failed): nothing is
// written, and a shard that had no error of its own reports OBEM_ERR_STATE
__global__ void sh_abort_kernel(StepCtl *ctl, obem_step_stats *stats)
{
    if (threadIdx.x != 0) return;
    ctl->abort = 1;
    if (stats->status == OBEM_OK) stats->status = OBEM_ERR_STATE;
    stats->n_after = stats->n_before;
}

__global__ void sh_set_id_kernel(uint32_t *next_id, uint32_t v)
{
    if (threadIdx.x == 0) *next_id = v;
}

int obem_launch_shard_commit(obem_ctx *c, const obem_state *stp, const float4 *E, uint32_t step, uint32_t id_base,
                             int commit, obem_step_stats *stats, cudaStream_t s)
{
    const obem_state st = *stp;
    const int cap = st.capacity;
    const int nblk = (cap + ST_THREADS - 1) / ST_THREADS;
    const GasDev g = step_gas(c);
    if (!commit) {
        sh_abort_kernel<<<1, 32, 0, s>>>(c->s_ctl, stats);
        OBEM_LAUNCH(c);
        return OBEM_OK;
    }
    sh_set_id_kernel<<<1, 32, 0, s>>>(st.next_id, id_base);
    write_kernel<<<nblk, ST_THREADS, 0, s>>>(st, g, E, step, c->s_prop, c->s_ionkey, c->s_keep,
                                             c->s_nsp, c->s_blk, c->s_ctl, c->o_pos, c->o_vel,
                                             c->o_id, c->o_birth, c->o_sp);
    OBEM_LAUNCH(c);
    commit_kernel<<<nblk, ST_THREADS, 0, s>>>(st, c->s_ctl, c->o_pos, c->o_vel, c->o_id, c->o_birth,
                                              c->o_sp);
    OBEM_LAUNCH(c);
    if (g.hit_on) {
        deposit_kernel<<<nblk, ST_THREADS, 0, s>>>(st, c->s_ctl, c->s_hit, (unsigned long long *)c->d_deposit);
        OBEM_LAUNCH(c);
    }
    finish_kernel<<<1, 32, 0, s>>>(st, c->s_ctl);
    OBEM_LAUNCH(c);
    moments_kernel<<<nblk, ST_THREADS, 0, s>>>(st, stats, c->s_mpart);
    moments_fold_kernel<<<1, 1024, 0, s>>>(st, c->s_mpart, stats);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}

int obem_launch_step(obem_ctx *c, const obem_state *stp, const float4 *E, uint32_t step,
                     obem_step_stats *stats, cudaStream_t s)
{
    const obem_state st = *stp;
    const int cap = st.capacity;
    const int nblk = (cap + ST_THREADS - 1) / ST_THREADS;
    GasDev g = c->gas;
    g.hit_on = (c->cfg.flags & OBEM_STEP_SURFACE_HITS) && c->np > 0 && c->d_tri9;
    if (g.hit_on) {
        g.tri9 = c->d_tri9;
        g.hstart = c->d_hstart;
        g.htri = c->d_htri;
        for (int k = 0; k < 3; ++k) { g.hlo[k] = c->h_hlo[k]; g.hdim[k] = c->h_hdim[k]; }
        g.hinv = c->h_hinv;
    }
    init_kernel<<<1, 32, 0, s>>>(stats, c->s_ctl, st);
    OBEM_LAUNCH(c);
    if (g.recomb_on) {
        if (g.rc2 > 0.f) {
            const double inv_h = 1.0 / (sqrt((double)g.rc2) * (1.0 + 1e-5));
            OBEM_CUDA(c, cudaMemsetAsync(c->ph_count, 0, sizeof(int32_t) * PH_BUCKETS, s));
            ph_count_kernel<<<nblk, ST_THREADS, 0, s>>>(st, step, inv_h, c->ph_bucket, c->ph_count);
            ph_blocksum_kernel<<<PH_NBLK, PH_BLK, 0, s>>>(c->ph_count, c->ph_bsum);
            ph_scan_sums_kernel<<<1, PH_BLK, 0, s>>>(c->ph_bsum);
            ph_scan_apply_kernel<<<PH_NBLK, PH_BLK, 0, s>>>(c->ph_count, c->ph_bsum, c->ph_start, c->ph_cursor);
            ph_scatter_kernel<<<nblk, ST_THREADS, 0, s>>>(st, c->ph_bucket, c->ph_cursor, c->ph_sorted);
            ph_query_kernel<<<nblk, ST_THREADS, 0, s>>>(st, g, inv_h, c->ph_start, c->ph_sorted, c->s_prop);
            OBEM_LAUNCH(c);
        } else {
            OBEM_CUDA(c, cudaMemsetAsync(c->s_prop, 0xFF, sizeof(u64) * (size_t)cap, s));
        }
        OBEM_CUDA(c, cudaMemsetAsync(c->s_ionkey, 0xFF, sizeof(u64) * (size_t)cap, s));
        resolve_kernel<<<nblk, ST_THREADS, 0, s>>>(st, c->s_prop, c->s_ionkey);
        OBEM_LAUNCH(c);
    }
    count_kernel<<<nblk, ST_THREADS, 0, s>>>(st, g, E, step, c->s_prop, c->s_ionkey, c->s_keep,
                                             c->s_nsp, c->s_blk, stats, c->s_ctl, c->s_hit);
    OBEM_LAUNCH(c);
    scan_kernel<<<1, 1024, 0, s>>>(st, c->s_blk, stats, c->s_ctl, cap < c->cap ? cap : c->cap);
    OBEM_LAUNCH(c);
    write_kernel<<<nblk, ST_THREADS, 0, s>>>(st, g, E, step, c->s_prop, c->s_ionkey, c->s_keep,
                                             c->s_nsp, c->s_blk, c->s_ctl, c->o_pos, c->o_vel,
                                             c->o_id, c->o_birth, c->o_sp);
    OBEM_LAUNCH(c);
    commit_kernel<<<nblk, ST_THREADS, 0, s>>>(st, c->s_ctl, c->o_pos, c->o_vel, c->o_id, c->o_birth,
                                              c->o_sp);
    OBEM_LAUNCH(c);
    if (g.hit_on) {
        deposit_kernel<<<nblk, ST_THREADS, 0, s>>>(st, c->s_ctl, c->s_hit, (unsigned long long *)c->d_deposit);
        OBEM_LAUNCH(c);
    }
    finish_kernel<<<1, 32, 0, s>>>(st, c->s_ctl);
    OBEM_LAUNCH(c);
    moments_kernel<<<nblk, ST_THREADS, 0, s>>>(st, stats, c->s_mpart);
    moments_fold_kernel<<<1, 1024, 0, s>>>(st, c->s_mpart, stats);
    OBEM_LAUNCH(c);
    if (c->prof_on) c->launches += 9 + (g.recomb_on ? 7 : 0) + (g.hit_on ? 1 : 0);
    return OBEM_OK;
}

// ====================================================================
// Batch of independent chambers.  Chamber c holds slots [seg_off[c],
// seg_off[c + 1]) of one concatenated state (multiples of OBEM_SEG_ALIGN, so
// each block of ST_THREADS slots belongs to one chamber), its first n[c]
// live.  The passes of the single step, each one launch for every chamber;
// a charge meets only charges of its own chamber, and its draws are keyed by
// its chamber's seed and its own id, so every chamber evolves exactly as it
// would alone.  The step index is read from the device and advanced by the
// last pass: the launch sequence can be captured once in a CUDA graph and
// replayed step after step.  If any chamber fails (capacity, trials), no
// chamber commits.

// chamber of the block, its first slot, its live charges; slot i's index in it
struct BtSlot {
    int c, off, n, li;
};
__device__ __forceinline__ BtSlot bt_slot(const StepBatch &B)
{
    BtSlot r;
    r.c = B.blk_cham[blockIdx.x];
    r.off = B.seg_off[r.c];
    r.n = B.n[r.c];
    r.li = blockIdx.x * ST_THREADS + threadIdx.x - r.off;
    return r;
}

__global__ void bt_init_kernel(StepBatch B)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) *B.abort = 0;
    if (c >= B.nb) return;
    memset(&B.stats[c], 0, sizeof(obem_step_stats));
    memset(&B.ctl[c], 0, sizeof(StepCtl));
    B.stats[c].n_before = B.n[c];
}

__device__ __forceinline__ uint32_t bt_hash(long long cx, long long cy, long long cz, int c)
{
    return (ph_hash(cx, cy, cz) ^ ((uint32_t)c * 0x9E3779B1u)) & (PH_BUCKETS - 1);
}

__global__ void bt_ph_count_kernel(const obem_state st, StepBatch B, double inv_h, int32_t *bucket_of, int32_t *count)
{
    const BtSlot q = bt_slot(B);
    if (q.li >= q.n) return;
    const int i = q.off + q.li;
    const uint32_t step = *B.step;
    const uint32_t b = st.birth[i];
    if (st.species[i] != OBEM_CATION || (b != 0u && b == step)) { bucket_of[i] = -1; return; }
    long long cx, cy, cz;
    ph_cell(reinterpret_cast<const float4 *>(st.pos_q)[i], inv_h, cx, cy, cz);
    const uint32_t h = bt_hash(cx, cy, cz, q.c);
    bucket_of[i] = (int32_t)h;
    atomicAdd(&count[h], 1);
}

__global__ void bt_ph_scatter_kernel(const obem_state st, StepBatch B, const int32_t *bucket_of, int32_t *cursor,
                                     int32_t *sorted)
{
    const BtSlot q = bt_slot(B);
    if (q.li >= q.n) return;
    const int i = q.off + q.li;
    const int32_t h = bucket_of[i];
    if (h < 0) return;
    sorted[atomicAdd(&cursor[h], 1)] = i;
}

// nearest eligible cation of the same chamber (keys carry slots: within a
// chamber, slot order is index order, so ties resolve as in a single step)
__global__ void bt_ph_query_kernel(const obem_state st, StepBatch B, GasDev g, double inv_h, const int32_t *start,
                                   const int32_t *sorted, u64 *prop)
{
    const BtSlot q = bt_slot(B);
    if (q.li >= q.n) return;
    const int i = q.off + q.li;
    u64 best = ~0ull;
    if (st.species[i] == OBEM_ELECTRON) {
        const float4 pe = reinterpret_cast<const float4 *>(st.pos_q)[i];
        long long cx, cy, cz;
        ph_cell(pe, inv_h, cx, cy, cz);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const uint32_t h = bt_hash(cx + dx, cy + dy, cz + dz, q.c);
                    for (int k = start[h]; k < start[h + 1]; ++k) {
                        const int c = sorted[k];
                        if (c < q.off || c >= q.off + q.n) continue;      // another chamber
                        const float4 pc = reinterpret_cast<const float4 *>(st.pos_q)[c];
                        const float ex = pe.x - pc.x, ey = pe.y - pc.y, ez = pe.z - pc.z;
                        const float d2 = ex * ex + ey * ey + ez * ez;
                        if (!(d2 <= g.rc2)) continue;
                        const u64 key = ((u64)__float_as_uint(d2) << 32) | (u64)(uint32_t)c;
                        if (key < best) best = key;
                    }
                }
    }
    prop[i] = best;
}

__global__ void bt_resolve_kernel(const obem_state st, StepBatch B, const u64 *prop, u64 *ionkey)
{
    const BtSlot q = bt_slot(B);
    if (q.li >= q.n) return;
    const int i = q.off + q.li;
    const u64 pr = prop[i];
    if (pr == ~0ull || st.species[i] != OBEM_ELECTRON) return;
    const uint32_t ion = (uint32_t)(pr & 0xFFFFFFFFu);
    atomicMin(&ionkey[ion], (pr & 0xFFFFFFFF00000000ull) | (u64)(uint32_t)i);
}

__global__ void __launch_bounds__(ST_THREADS)
bt_count_kernel(const obem_state st, StepBatch B, GasDev g, const float4 *E, const u64 *prop, const u64 *ionkey,
                int32_t *keep, int32_t *nsp, int32_t *blk)
{
    __shared__ long long sh[ST_THREADS / 32];
    const BtSlot q = bt_slot(B);
    const uint32_t step = *B.step;
    int kp = 0, ns = 0, absorbed = 0, attached = 0, coll = 0, rec = 0, ovf = 0;
    long long trials = 0;
    if (q.li < q.n) {
        const int i = q.off + q.li;
        const uint8_t s = st.species[i];
        if (recombined(i, s, prop, ionkey, g.recomb_on)) {
            rec = (s == OBEM_CATION);
        } else {
            const float4 pq = reinterpret_cast<const float4 *>(st.pos_q)[i];
            const float4 vv = reinterpret_cast<const float4 *>(st.vel)[i];
            const float4 e = E[i];
            float3 p = make_float3(pq.x, pq.y, pq.z), v = make_float3(vv.x, vv.y, vv.z);
            uint8_t sp = s;
            FlightOut fo = {0, 0, 0, 0, 0, 0, -1};
            fly<false>(g, B.cham[q.c], st.id[i], step, p, v, sp, make_float3(e.x, e.y, e.z), fo, NULL, NULL, NULL,
                       NULL, NULL, 0, 0u);
            kp = !fo.dead;
            ns = fo.nsp;
            absorbed = fo.dead;
            attached = fo.attached;
            coll = fo.collisions;
            trials = fo.trials;
            ovf = fo.overflow;
        }
        keep[i] = kp;
        nsp[i] = ns;
    }
    obem_step_stats *stt = &B.stats[q.c];
    long long t;
    t = block_sum<long long>(kp, sh);
    if (threadIdx.x == 0) blk[2 * blockIdx.x] = (int32_t)t;
    t = block_sum<long long>(ns, sh);
    if (threadIdx.x == 0) blk[2 * blockIdx.x + 1] = (int32_t)t;
    t = block_sum<long long>(absorbed, sh);
    if (threadIdx.x == 0 && t) atomicAdd(&stt->absorbed, (int)t);
    t = block_sum<long long>(attached, sh);
    if (threadIdx.x == 0 && t) atomicAdd(&stt->attached, (int)t);
    t = block_sum<long long>(coll, sh);
    if (threadIdx.x == 0 && t) atomicAdd(&stt->collisions, (int)t);
    t = block_sum<long long>(rec, sh);
    if (threadIdx.x == 0 && t) atomicAdd(&stt->recombined_pairs, (int)t);
    t = block_sum<long long>(trials, sh);
    if (threadIdx.x == 0 && t) atomicAdd((unsigned long long *)&stt->trials, (unsigned long long)t);
    t = block_sum<long long>(ovf, sh);
    if (threadIdx.x == 0 && t) atomicOr(&B.ctl[q.c].trial_overflow, 1);
}

// one block per chamber: exclusive scan of its blocks' (keep, spawn) totals,
// capacity and trial checks
__global__ void bt_scan_kernel(StepBatch B, int32_t *blk)
{
    __shared__ int32_t sk[1024], ss[1024];
    __shared__ int32_t carry_k, carry_s;
    const int c = blockIdx.x;
    const int n = B.n[c];
    const int b0 = B.seg_off[c] / ST_THREADS;
    const int nb = (n + ST_THREADS - 1) / ST_THREADS;
    const int cap = B.seg_off[c + 1] - B.seg_off[c];
    if (threadIdx.x == 0) { carry_k = 0; carry_s = 0; }
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        const int b = c0 + threadIdx.x;
        const int vk = b < nb ? blk[2 * (b0 + b)] : 0;
        const int vs = b < nb ? blk[2 * (b0 + b) + 1] : 0;
        sk[threadIdx.x] = vk;
        ss[threadIdx.x] = vs;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int ak = threadIdx.x >= o ? sk[threadIdx.x - o] : 0;
            const int as = threadIdx.x >= o ? ss[threadIdx.x - o] : 0;
            __syncthreads();
            sk[threadIdx.x] += ak;
            ss[threadIdx.x] += as;
            __syncthreads();
        }
        if (b < nb) {
            blk[2 * (b0 + b)] = carry_k + sk[threadIdx.x] - vk;
            blk[2 * (b0 + b) + 1] = carry_s + ss[threadIdx.x] - vs;
        }
        __syncthreads();
        if (threadIdx.x == 1023) { carry_k += sk[1023]; carry_s += ss[1023]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        StepCtl *ctl = &B.ctl[c];
        obem_step_stats *stt = &B.stats[c];
        const long long total = (long long)carry_k + 2ll * carry_s;
        ctl->n_keep = carry_k;
        ctl->n_spawn = carry_s;
        stt->spawned_pairs = carry_s;
        stt->required_capacity = total > 0x7fffffff ? 0x7fffffff : (int)total;
        if (ctl->trial_overflow) {
            stt->status = OBEM_ERR_TRIALS;
            atomicOr(B.abort, 1);
        } else if (total > cap) {
            stt->status = OBEM_ERR_CAPACITY;
            atomicOr(B.abort, 1);
        }
    }
}

__global__ void __launch_bounds__(ST_THREADS)
bt_write_kernel(const obem_state st, StepBatch B, GasDev g, const float4 *E, const u64 *prop, const u64 *ionkey,
                const int32_t *keep, const int32_t *nsp, const int32_t *blk, float4 *o_pos, float4 *o_vel,
                uint32_t *o_id, uint32_t *o_birth, uint8_t *o_sp)
{
    __shared__ int32_t wk[ST_THREADS / 32], ws[ST_THREADS / 32];
    if (*B.abort) return;
    const BtSlot q = bt_slot(B);
    const uint32_t step = *B.step;
    const int i = q.off + q.li;
    int kp = 0, ns = 0;
    if (q.li < q.n) { kp = keep[i]; ns = nsp[i]; }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ik = kp, is = ns;
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, ik, o);
        const int b = __shfl_up_sync(0xffffffffu, is, o);
        if (lane >= o) { ik += a; is += b; }
    }
    if (lane == 31) { wk[warp] = ik; ws[warp] = is; }
    __syncthreads();
    int pk_ = 0, ps_ = 0;
    for (int w = 0; w < warp; ++w) { pk_ += wk[w]; ps_ += ws[w]; }
    if (q.li >= q.n || (!kp && !ns)) return;
    const int out_keep = blk[2 * blockIdx.x] + pk_ + ik - kp;
    const int out_spawn = blk[2 * blockIdx.x + 1] + ps_ + is - ns;
    const uint8_t s = st.species[i];
    const float4 pq = reinterpret_cast<const float4 *>(st.pos_q)[i];
    const float4 vv = reinterpret_cast<const float4 *>(st.vel)[i];
    const float4 e = E[i];
    float3 p = make_float3(pq.x, pq.y, pq.z), v = make_float3(vv.x, vv.y, vv.z);
    uint8_t sp = s;
    FlightOut fo = {0, 0, 0, 0, 0, 0, -1};
    const int sbase = q.off + B.ctl[q.c].n_keep + 2 * out_spawn;
    const uint32_t id_base = B.next_id[q.c] + (uint32_t)(2 * out_spawn);
    fly<true>(g, B.cham[q.c], st.id[i], step, p, v, sp, make_float3(e.x, e.y, e.z), fo, o_pos, o_vel, o_id,
              o_birth, o_sp, sbase, id_base);
    if (kp) {
        const int o = q.off + out_keep;
        o_pos[o] = make_float4(p.x, p.y, p.z, pq.w);
        o_vel[o] = make_float4(v.x, v.y, v.z, vv.w);
        o_id[o] = st.id[i];
        o_birth[o] = st.birth[i];
        o_sp[o] = sp;                    // after the flight (attachment makes an anion)
    }
}

__global__ void bt_commit_kernel(const obem_state st, StepBatch B, const float4 *o_pos, const float4 *o_vel,
                                 const uint32_t *o_id, const uint32_t *o_birth, const uint8_t *o_sp)
{
    if (*B.abort) return;
    const BtSlot q = bt_slot(B);
    const StepCtl &ctl = B.ctl[q.c];
    if (q.li >= ctl.n_keep + 2 * ctl.n_spawn) return;
    const int i = q.off + q.li;
    reinterpret_cast<float4 *>(st.pos_q)[i] = o_pos[i];
    reinterpret_cast<float4 *>(st.vel)[i] = o_vel[i];
    st.id[i] = o_id[i];
    st.birth[i] = o_birth[i];
    st.species[i] = o_sp[i];
}

// per chamber: new counts (or, when any chamber failed, the chambers that did
// not fail report OBEM_ERR_STATE: nothing was committed); the step index
// advances when the batch committed
__global__ void bt_finish_kernel(StepBatch B)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool ab = *B.abort != 0;
    if (c == 0 && !ab) *B.step += 1u;
    if (c >= B.nb) return;
    obem_step_stats *stt = &B.stats[c];
    if (ab) {
        if (stt->status == OBEM_OK) stt->status = OBEM_ERR_STATE;
        stt->n_after = stt->n_before;
        return;
    }
    const StepCtl &ctl = B.ctl[c];
    B.n[c] = ctl.n_keep + 2 * ctl.n_spawn;
    B.next_id[c] = B.next_id[c] + (uint32_t)(2 * ctl.n_spawn);
    stt->n_after = B.n[c];
}

__global__ void __launch_bounds__(ST_THREADS)
bt_moments_kernel(const obem_state st, StepBatch B, double *part)
{
    const BtSlot q = bt_slot(B);
    if (q.li - (int)threadIdx.x >= q.n) return;          // a block past the chamber's charges
    moments_block(st, q.off + q.li, q.li < q.n, &B.stats[q.c], part + (size_t)NMOM * blockIdx.x);
}

// one block per chamber: its blocks' partial sums in block order
__global__ void __launch_bounds__(1024) bt_moments_fold_kernel(StepBatch B, const double *part)
{
    const int c = blockIdx.x;
    const int b0 = B.seg_off[c] / ST_THREADS;
    moments_fold(part + (size_t)NMOM * b0, (B.n[c] + ST_THREADS - 1) / ST_THREADS, &B.stats[c]);
}

// The whole batched step on stream s.  Scratch (BtScratch) is sized for the
// batch's slots; E holds the field at every live slot.
int obem_launch_step_batch(obem_ctx *c, const obem_state *stp, const StepBatch &B, const BtScratch &W,
                           const float4 *E, cudaStream_t s)
{
    const obem_state st = *stp;
    const int slots = st.capacity;
    const int nblk = slots / ST_THREADS;
    GasDev g = c->gas;
    g.hit_on = 0;
    const int cb = (B.nb + 255) / 256;
    bt_init_kernel<<<cb, 256, 0, s>>>(B);
    OBEM_LAUNCH(c);
    if (g.recomb_on) {
        if (g.rc2 > 0.f) {
            const double inv_h = 1.0 / (sqrt((double)g.rc2) * (1.0 + 1e-5));
            OBEM_CUDA(c, cudaMemsetAsync(W.ph_count, 0, sizeof(int32_t) * PH_BUCKETS, s));
            bt_ph_count_kernel<<<nblk, ST_THREADS, 0, s>>>(st, B, inv_h, W.ph_bucket, W.ph_count);
            ph_blocksum_kernel<<<PH_NBLK, PH_BLK, 0, s>>>(W.ph_count, W.ph_bsum);
            ph_scan_sums_kernel<<<1, PH_BLK, 0, s>>>(W.ph_bsum);
            ph_scan_apply_kernel<<<PH_NBLK, PH_BLK, 0, s>>>(W.ph_count, W.ph_bsum, W.ph_start, W.ph_cursor);
            bt_ph_scatter_kernel<<<nblk, ST_THREADS, 0, s>>>(st, B, W.ph_bucket, W.ph_cursor, W.ph_sorted);
            bt_ph_query_kernel<<<nblk, ST_THREADS, 0, s>>>(st, B, g, inv_h, W.ph_start, W.ph_sorted, W.prop);
            OBEM_LAUNCH(c);
        } else {
            OBEM_CUDA(c, cudaMemsetAsync(W.prop, 0xFF, sizeof(u64) * (size_t)slots, s));
        }
        OBEM_CUDA(c, cudaMemsetAsync(W.ionkey, 0xFF, sizeof(u64) * (size_t)slots, s));
        bt_resolve_kernel<<<nblk, ST_THREADS, 0, s>>>(st, B, W.prop, W.ionkey);
        OBEM_LAUNCH(c);
    }
    bt_count_kernel<<<nblk, ST_THREADS, 0, s>>>(st, B, g, E, W.prop, W.ionkey, W.keep, W.nsp, W.blk);
    OBEM_LAUNCH(c);
    bt_scan_kernel<<<B.nb, 1024, 0, s>>>(B, W.blk);
    OBEM_LAUNCH(c);
    bt_write_kernel<<<nblk, ST_THREADS, 0, s>>>(st, B, g, E, W.prop, W.ionkey, W.keep, W.nsp, W.blk, W.o_pos,
                                                W.o_vel, W.o_id, W.o_birth, W.o_sp);
    OBEM_LAUNCH(c);
    bt_commit_kernel<<<nblk, ST_THREADS, 0, s>>>(st, B, W.o_pos, W.o_vel, W.o_id, W.o_birth, W.o_sp);
    OBEM_LAUNCH(c);
    bt_finish_kernel<<<cb, 256, 0, s>>>(B);
    OBEM_LAUNCH(c);
    bt_moments_kernel<<<nblk, ST_THREADS, 0, s>>>(st, B, W.mpart);
    bt_moments_fold_kernel<<<B.nb, 1024, 0, s>>>(B, W.mpart);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}
