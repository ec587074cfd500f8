/*
 * obem_oracle.c -- plain, slow, CPU reference ("oracle") for the OuroborosBEM
 * field + tracking-step method (arXiv 2110.09214).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the test-suite, the smoke check and the CPU-baseline leg of the bench
 * load it.  It shares no source with the CUDA library.
 *
 * Floating point:
 *   - geometry, panel integrals, the panel field, the N-body field, the BEM
 *     matrix and its Gaussian elimination are FP64;
 *   - the tracking step (flight, null-collision trials, ionisation, attachment,
 *     recombination distances) is computed in IEEE binary32 with one rounding
 *     per basic operation (build with -ffp-contract=off, no fast-math), because
 *     every integer decision of the step (collision process, spawn count,
 *     recombination partner) must be taken in the precision of the kernel.
 *
 * Every function cites the passage of the paper it restates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018, SI */
#define OR_E    1.602176634e-19
#define OR_ME   9.1093837015e-31
#define OR_EPS0 8.8541878128e-12
#define OR_KB   1.380649e-23
#define OR_AMU  1.66053906660e-27
#define OR_PI   3.14159265358979323846
#define OR_KC   (1.0 / (4.0 * OR_PI * OR_EPS0))

/* ------------------------------------------------------------------------- */
/* small FP64 vector helpers                                                  */
/* ------------------------------------------------------------------------- */
static double dot3(const double *a, const double *b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1]*b[2] - a[2]*b[1];
    c[1] = a[2]*b[0] - a[0]*b[2];
    c[2] = a[0]*b[1] - a[1]*b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* Geometry of a flat triangular cell (Sec. 2.2: flat cells, centroid
 * collocation, unit normal).  v = 9 doubles (v0, v1, v2).  The normal is
 * (v1-v0)x(v2-v0) normalised: it points from medium 1 (eps_minus) to medium 2
 * (eps_plus), the orientation used by Eq. (fldinterf1/2) and (NBC). */
void or_tri_geometry(const double *v, double *centroid, double *normal, double *area)
{
    double e1[3], e2[3], nn[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = v[3 + k] - v[k];
        e2[k] = v[6 + k] - v[k];
        centroid[k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0;
    }
    cross3(e1, e2, nn);
    double a2 = norm3(nn);
    for (int k = 0; k < 3; ++k) normal[k] = nn[k] / a2;
    *area = 0.5 * a2;
}

/* Log of the line integral of 1/R along one edge, written so that no
 * difference of nearly equal numbers is formed (products (R+l)(R-l) = R0^2 are
 * the same at both ends of the edge). */
static double edge_log(double lm, double lp, double Rm, double Rp, double R0sq)
{
    if (lm >= 0.0) return log((Rp + lp) / (Rm + lm));
    if (lp <= 0.0) return log((Rm - lm) / (Rp - lp));
    return log((Rp + lp) * (Rm - lm) / R0sq);
}

/*
 * Closed-form surface integrals of a uniform unit density over a flat
 * triangle, at observation point r (Sec. 2.2 states that the cell integrals of
 * Eqs. (BEMpot), (BEMfld), (BEM2), (BEM3) are evaluated analytically but does
 * not print them; this is the standard edge decomposition of the potential of
 * a planar polygon (Wilton et al. 1984) with the solid angle of Van Oosterom &
 * Strackee 1983):
 *
 *   phi(r) = int_T dA' / |r - r'|
 *          = sum_edges p0_i L_i - h * Omega
 *   F(r)   = int_T (r - r') / |r - r'|^3 dA'
 *          = Omega n + sum_edges u_i L_i
 *
 * with h = (r - v0).n, u_i the outward in-plane unit normal of edge i, p0_i the
 * signed in-plane distance from the projection of r to edge i (positive
 * inside), L_i = ln((R+ + l+)/(R- + l-)) the edge line integral of 1/R, and
 * Omega the solid angle of the triangle seen from r, signed like h.
 * In the plane of the cell (h = 0) the normal part is the principal value,
 * i.e. the mean of the two one-sided limits -+ 2pi of Eq. (fldinterf1/2), 0.
 */
void or_tri_integrals(const double *v, const double *r, double *phi, double *F)
{
    double e1[3], e2[3], nn[3], n[3], a[3][3], R[3];
    for (int k = 0; k < 3; ++k) { e1[k] = v[3 + k] - v[k]; e2[k] = v[6 + k] - v[k]; }
    cross3(e1, e2, nn);
    double a2 = norm3(nn);                 /* twice the area */
    for (int k = 0; k < 3; ++k) n[k] = nn[k] / a2;
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) a[i][k] = v[3 * i + k] - r[k];
        R[i] = norm3(a[i]);
    }
    double h = -dot3(a[0], n);
    double phis = 0.0, Fin[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        double ed[3], lhat[3], uhat[3];
        for (int k = 0; k < 3; ++k) ed[k] = v[3 * j + k] - v[3 * i + k];
        double len = norm3(ed);
        for (int k = 0; k < 3; ++k) lhat[k] = ed[k] / len;
        cross3(lhat, n, uhat);
        double lm = dot3(a[i], lhat), lp = dot3(a[j], lhat);
        double p0 = dot3(a[i], uhat);
        double R0sq = p0 * p0 + h * h;
        double L = edge_log(lm, lp, R[i], R[j], R0sq);
        if (p0 != 0.0) phis += p0 * L;
        for (int k = 0; k < 3; ++k) Fin[k] += uhat[k] * L;
    }
    double D = R[0] * R[1] * R[2] + dot3(a[0], a[1]) * R[2] + dot3(a[0], a[2]) * R[1]
             + dot3(a[1], a[2]) * R[0];
    double Om = (h == 0.0) ? 0.0 : 2.0 * atan2(a2 * h, D);
    *phi = phis - h * Om;
    for (int k = 0; k < 3; ++k) F[k] = Fin[k] + Om * n[k];
}

/* Potential and field of all panels at nt points, Eqs. (BEM2), (BEM3):
 *   V(r) = k_C sum_j sigma_j phi_j(r),  E(r) = k_C sum_j sigma_j F_j(r). */
void or_panel_field(int np, const double *tri, const double *sigma, int nt,
                    const double *pts, double *E, double *V)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nt; ++t) {
        double ex = 0, ey = 0, ez = 0, vv = 0;
        for (int j = 0; j < np; ++j) {
            double phi, F[3];
            or_tri_integrals(tri + 9 * (size_t)j, pts + 3 * (size_t)t, &phi, F);
            ex += sigma[j] * F[0]; ey += sigma[j] * F[1]; ez += sigma[j] * F[2];
            vv += sigma[j] * phi;
        }
        E[3 * t] = OR_KC * ex; E[3 * t + 1] = OR_KC * ey; E[3 * t + 2] = OR_KC * ez;
        if (V) V[t] = OR_KC * vv;
    }
}

/* Coulomb field of point charges, Eq. (nbody):
 *   E(r_t) = k_C sum_{p != t} q_p (r_t - r_p) / |r_t - r_p|^3
 * src = [x,y,z,q] per source.  self_exclude: target t and source t are the same
 * charge and that pair is skipped.  soft > 0 replaces |r|^2 by |r|^2 + soft^2
 * (Plummer); soft == 0 is the paper's sum, in which pairs at zero distance are
 * skipped (the sum is undefined there). */
void or_nbody_field(int nt, const double *pts, int ns, const double *src,
                    int self_exclude, double soft, double *E, double *V)
{
    double s2 = soft * soft;
#pragma omp parallel for schedule(static)
    for (int t = 0; t < nt; ++t) {
        double ex = 0, ey = 0, ez = 0, vv = 0;
        const double *r = pts + 3 * (size_t)t;
        for (int p = 0; p < ns; ++p) {
            if (self_exclude && p == t) continue;
            const double *s = src + 4 * (size_t)p;
            double dx = r[0] - s[0], dy = r[1] - s[1], dz = r[2] - s[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0 && s2 == 0.0) continue;
            r2 += s2;
            double ir = 1.0 / sqrt(r2);
            double w = s[3] * ir * ir * ir;
            ex += w * dx; ey += w * dy; ez += w * dz;
            vv += s[3] * ir;
        }
        E[3 * t] = OR_KC * ex; E[3 * t + 1] = OR_KC * ey; E[3 * t + 2] = OR_KC * ez;
        if (V) V[t] = OR_KC * vv;
    }
}

/* ------------------------------------------------------------------------- */
/* Derivatives of the field (backward / adjoint evaluation of Eqs. (BEM2),    */
/* (BEM3), (nbody)).  The paper does not differentiate its field; these are   */
/* the derivatives of the closed forms above, written out.                    */
/* ------------------------------------------------------------------------- */

/* Gradient, with respect to the observation point r, of the edge term
 * L = ln((R+ + l+)/(R- + l-)) of or_tri_integrals.  With a = v - r for either
 * end, l = a.lhat, and w the part of a perpendicular to the edge (the same
 * vector at both ends):  grad(R + l) = -(a/R + lhat) and
 * (a/R + lhat)/(R + l) = lhat/R + w/(R (R + l)), hence
 *   grad L = lhat (1/R- - 1/R+) + w (g(R-, l-) - g(R+, l+)),  g = 1/(R (R + l)).
 * R + l is formed without cancellation in each of the three cases that
 * edge_log distinguishes (foot of r before, past, or on the edge). */
static void edge_log_grad(const double *lhat, const double *w, double lm, double lp,
                          double Rm, double Rp, double R0sq, double *g)
{
    double cw;
    if (lm >= 0.0)
        cw = 1.0 / (Rm * (Rm + lm)) - 1.0 / (Rp * (Rp + lp));
    else if (lp <= 0.0)   /* the same edge walked backwards: L = ln((R- - l-)/(R+ - l+)) */
        cw = -(1.0 / (Rm * (Rm - lm)) - 1.0 / (Rp * (Rp - lp)));
    else                  /* 1/(R- (R- + l-)) = (R- - l-)/(R- R0^2) */
        cw = (Rm - lm) / (Rm * R0sq) - 1.0 / (Rp * (Rp + lp));
    double cl = 1.0 / Rm - 1.0 / Rp;
    for (int k = 0; k < 3; ++k) g[k] = cl * lhat[k] + cw * w[k];
}

/*
 * Jacobian J[a][b] = dF_a/dr_b of F(r) = int_T (r - r')/|r - r'|^3 dA' (unit
 * density), row-major.  From F = Omega n + sum_edges u_i L_i:
 *   J = n (grad Omega)^T + sum_i u_i (grad L_i)^T.
 * The gradient of the solid angle of a flat polygon is the Biot-Savart line
 * integral of a unit current around its boundary; for the straight edge from
 * v_i to v_j it is
 *   (lhat x w) / R0^2 * (l+/R+ - l-/R-),
 * and when l- and l+ have the same sign the bracket is rewritten as
 *   R0^2 (l+^2 - l-^2) / ((l+ R- + l- R+) R- R+)
 * so that R0^2 cancels (no loss of digits near the edge's line).  F = -grad
 * phi, so J is symmetric, and off the triangle trace(J) = 0 (Laplace).
 * Defined for r off the closed triangle.
 */
void or_tri_jacobian(const double *v, const double *r, double *J)
{
    double e1[3], e2[3], nn[3], n[3], a[3][3], R[3];
    for (int k = 0; k < 3; ++k) { e1[k] = v[3 + k] - v[k]; e2[k] = v[6 + k] - v[k]; }
    cross3(e1, e2, nn);
    double a2 = norm3(nn);
    for (int k = 0; k < 3; ++k) n[k] = nn[k] / a2;
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) a[i][k] = v[3 * i + k] - r[k];
        R[i] = norm3(a[i]);
    }
    double h = -dot3(a[0], n);
    double gOm[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 9; ++k) J[k] = 0.0;
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        double ed[3], lhat[3], uhat[3], w[3], gL[3], lw[3];
        for (int k = 0; k < 3; ++k) ed[k] = v[3 * j + k] - v[3 * i + k];
        double len = norm3(ed);
        for (int k = 0; k < 3; ++k) lhat[k] = ed[k] / len;
        cross3(lhat, n, uhat);
        double lm = dot3(a[i], lhat), lp = dot3(a[j], lhat);
        for (int k = 0; k < 3; ++k) w[k] = a[i][k] - lm * lhat[k];
        double p0 = dot3(a[i], uhat);
        double R0sq = p0 * p0 + h * h;
        edge_log_grad(lhat, w, lm, lp, R[i], R[j], R0sq, gL);
        for (int ia = 0; ia < 3; ++ia)
            for (int ib = 0; ib < 3; ++ib) J[3 * ia + ib] += uhat[ia] * gL[ib];
        cross3(lhat, w, lw);
        double c;
        if (lm * lp > 0.0)
            c = (lp * lp - lm * lm) / ((lp * R[i] + lm * R[j]) * R[i] * R[j]);
        else
            c = (lp / R[j] - lm / R[i]) / R0sq;
        for (int k = 0; k < 3; ++k) gOm[k] += c * lw[k];
    }
    for (int ia = 0; ia < 3; ++ia)
        for (int ib = 0; ib < 3; ++ib) J[3 * ia + ib] += n[ia] * gOm[ib];
}

/* Jacobian of the total field at nt points, d E / d r (row-major 3x3 each):
 *   k_C sum_j sigma_j J_j(r) + k_C sum_{p != t} q_p (I/d^3 - 3 d d^T/d^5),
 * d = r - r_p (the derivative of Eq. (nbody)'s pair term); pairs at zero
 * distance are skipped as in or_nbody_field.  tri/sigma or src may be empty. */
void or_field_jacobian(int np, const double *tri, const double *sigma, int nt, const double *pts,
                       int ns, const double *src, int self_exclude, double *Jout)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nt; ++t) {
        const double *r = pts + 3 * (size_t)t;
        double acc[9] = {0};
        for (int j = 0; j < np; ++j) {
            double Jj[9];
            or_tri_jacobian(tri + 9 * (size_t)j, r, Jj);
            for (int k = 0; k < 9; ++k) acc[k] += sigma[j] * Jj[k];
        }
        for (int p = 0; p < ns; ++p) {
            if (self_exclude && p == t) continue;
            const double *s = src + 4 * (size_t)p;
            double d[3] = {r[0] - s[0], r[1] - s[1], r[2] - s[2]};
            double d2 = dot3(d, d);
            if (d2 == 0.0) continue;
            double id = 1.0 / sqrt(d2), id3 = id * id * id, id5 = id3 * id * id;
            for (int ia = 0; ia < 3; ++ia)
                for (int ib = 0; ib < 3; ++ib)
                    acc[3 * ia + ib] += s[3] * ((ia == ib ? id3 : 0.0) - 3.0 * d[ia] * d[ib] * id5);
        }
        for (int k = 0; k < 9; ++k) Jout[9 * (size_t)t + k] = OR_KC * acc[k];
    }
}

/*
 * Backward (vector-Jacobian product) of the field evaluation
 *   E_t = k_C sum_j sigma_j F_j(x_t) + k_C sum_{p != t} q_p (x_t - y_p)/|x_t - y_p|^3
 *   V_t = k_C sum_j sigma_j phi_j(x_t) + k_C sum_{p != t} q_p / |x_t - y_p|
 * for L with dL/d(E_t, V_t) = g_t = (gE_t, gV_t) (g: nt x 4):
 *   dL/dsigma_j = k_C sum_t gE_t . F_j(x_t) + gV_t phi_j(x_t)
 *   dL/dx_t     = (dE_t/dx_t)^T gE_t - gV_t E_t          (grad V = -E)
 *   dL/dy_p     = k_C q_p sum_t -T(d)^T gE_t + gV_t d/|d|^3,  d = x_t - y_p
 *   dL/dq_p     = k_C sum_t gE_t . d/|d|^3 + gV_t/|d|
 * with T(d) = I/|d|^3 - 3 d d^T/|d|^5.  Any output may be NULL.  dpts is
 * nt x 3, dsrc is ns x 4 (position gradient, charge gradient).
 */
void or_field_backward(int np, const double *tri, const double *sigma, int nt, const double *pts,
                       int ns, const double *src, int self_exclude, const double *g,
                       double *dsigma, double *dpts, double *dsrc)
{
    if (dsigma) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int j = 0; j < np; ++j) {
            double acc = 0.0;
            for (int t = 0; t < nt; ++t) {
                double phi, F[3];
                or_tri_integrals(tri + 9 * (size_t)j, pts + 3 * (size_t)t, &phi, F);
                const double *gt = g + 4 * (size_t)t;
                acc += gt[0] * F[0] + gt[1] * F[1] + gt[2] * F[2] + gt[3] * phi;
            }
            dsigma[j] = OR_KC * acc;
        }
    }
    if (dpts) {
        double *J = (double *)malloc(sizeof(double) * 9 * (size_t)(nt > 0 ? nt : 1));
        double *E = (double *)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
        double *E2 = (double *)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
        or_field_jacobian(np, tri, sigma, nt, pts, ns, src, self_exclude, J);
        for (int k = 0; k < 3 * nt; ++k) E[k] = 0.0;
        if (np > 0) or_panel_field(np, tri, sigma, nt, pts, E, NULL);
        if (ns > 0) {
            or_nbody_field(nt, pts, ns, src, self_exclude, 0.0, E2, NULL);
            for (int k = 0; k < 3 * nt; ++k) E[k] += E2[k];
        }
        for (int t = 0; t < nt; ++t) {
            const double *gt = g + 4 * (size_t)t;
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int a = 0; a < 3; ++a) s += J[9 * (size_t)t + 3 * a + b] * gt[a];
                dpts[3 * (size_t)t + b] = s - gt[3] * E[3 * (size_t)t + b];
            }
        }
        free(J); free(E); free(E2);
    }
    if (dsrc) {
#pragma omp parallel for schedule(static)
        for (int p = 0; p < ns; ++p) {
            const double *s = src + 4 * (size_t)p;
            double gy[3] = {0, 0, 0}, gq = 0.0;
            for (int t = 0; t < nt; ++t) {
                if (self_exclude && p == t) continue;
                const double *x = pts + 3 * (size_t)t, *gt = g + 4 * (size_t)t;
                double d[3] = {x[0] - s[0], x[1] - s[1], x[2] - s[2]};
                double d2 = dot3(d, d);
                if (d2 == 0.0) continue;
                double id = 1.0 / sqrt(d2), id3 = id * id * id, id5 = id3 * id * id;
                double dg = dot3(d, gt);
                for (int b = 0; b < 3; ++b)
                    gy[b] += -(gt[b] * id3 - 3.0 * d[b] * dg * id5) + gt[3] * d[b] * id3;
                gq += dg * id3 + gt[3] * id;
            }
            for (int b = 0; b < 3; ++b) dsrc[4 * (size_t)p + b] = OR_KC * s[3] * gy[b];
            dsrc[4 * (size_t)p + 3] = OR_KC * gq;
        }
    }
}

/* Trilinear interpolation on a regular grid (the static field map of
 * Sec. 2.4): values[((k * ny) + j) * nx + i][nc] at lo + (i, j, k) * step;
 * a point outside the grid's box is moved to the nearest point of the box.
 * Within a grid cell with fractional coordinates (tx, ty, tz):
 *   f = sum over the 8 corners of prod_a (t_a or 1 - t_a) * value(corner). */
void or_trilinear(int nx, int ny, int nz, const double *lo, const double *step, int nc, const double *values,
                  int n, const double *pts, double *out)
{
    const int dims[3] = {nx, ny, nz};
    for (int p = 0; p < n; ++p) {
        int i0[3];
        double t[3];
        for (int a = 0; a < 3; ++a) {
            double f = (pts[3 * (size_t)p + a] - lo[a]) / step[a];
            if (f < 0.0) f = 0.0;
            if (f > dims[a] - 1) f = dims[a] - 1;
            i0[a] = (int)floor(f);
            if (i0[a] > dims[a] - 2) i0[a] = dims[a] - 2;
            t[a] = f - i0[a];
        }
        for (int c = 0; c < nc; ++c) out[(size_t)p * nc + c] = 0.0;
        for (int corner = 0; corner < 8; ++corner) {
            const int dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
            const double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
            const size_t node = ((size_t)(i0[2] + dz) * ny + (i0[1] + dy)) * nx + (i0[0] + dx);
            for (int c = 0; c < nc; ++c) out[(size_t)p * nc + c] += w * values[node * nc + c];
        }
    }
}

/*
 * Approximate N-body field (Sec. 3.2.4, the nearest-neighbour "NN" option):
 * the exact Coulomb sum of Eq. (nbody) over the charges close to a particle,
 * the charge centres of the farther ones.  The paper describes it in one
 * sentence; the reading here:
 *   - cubic cells of edge W / G, W the largest extent of the charges'
 *     bounding box (G x G x G cells cover it); the cell of a charge is
 *     floor((x - lo) * (G / W)) per axis in binary32 (one rounding per
 *     operation; clamped to 0..G-1), so that both implementations put a
 *     charge in the same cell;
 *   - near: the exact (softened) pair sum over the charges of the 27 cells
 *     around the particle's cell, itself excluded;
 *   - far: every other cell contributes its positive and its negative charge
 *     separately, each as the total charge placed at its charge-weighted
 *     centre (one "centre of charges" per sign keeps a neutral cell of
 *     electrons and ions meaningful).
 * src: [x, y, z, q] per charge (binary32 values); E: [n][3], FP64.
 */
void or_nbody_nn(int n, const double *src, int G, double soft, double *E)
{
    if (n <= 0) return;
    float lo[3], hi[3], inv[3], wmax = 0.0f;
    for (int a = 0; a < 3; ++a) {
        lo[a] = hi[a] = (float)src[a];
        for (int i = 1; i < n; ++i) {
            float x = (float)src[4 * (size_t)i + a];
            if (x < lo[a]) lo[a] = x;
            if (x > hi[a]) hi[a] = x;
        }
        float w = hi[a] - lo[a];
        if (w > wmax) wmax = w;
    }
    if (!(wmax > 0.0f)) wmax = 1.0f;
    for (int a = 0; a < 3; ++a) inv[a] = (float)G / wmax;
    const int ncell = G * G * G;
    int *cell = (int *)malloc(sizeof(int) * (size_t)n);
    int *cc = (int *)malloc(sizeof(int) * 3 * (size_t)n);
    double *agg = (double *)calloc((size_t)ncell * 8, sizeof(double));   /* [cell][sign][x y z q] */
    for (int i = 0; i < n; ++i) {
        int c3[3];
        for (int a = 0; a < 3; ++a) {
            float x = (float)src[4 * (size_t)i + a];
            float t = (x - lo[a]) * inv[a];
            int k = (int)floorf(t);
            if (k < 0) k = 0;
            if (k > G - 1) k = G - 1;
            c3[a] = k;
            cc[3 * (size_t)i + a] = k;
        }
        int c = (c3[2] * G + c3[1]) * G + c3[0];
        cell[i] = c;
        double q = src[4 * (size_t)i + 3];
        double *ag = agg + (size_t)c * 8 + (q >= 0.0 ? 0 : 4);
        for (int a = 0; a < 3; ++a) ag[a] += q * src[4 * (size_t)i + a];
        ag[3] += q;
    }
    for (int c = 0; c < 2 * ncell; ++c) {
        double *ag = agg + (size_t)c * 4;
        if (ag[3] != 0.0) for (int a = 0; a < 3; ++a) ag[a] /= ag[3];
    }
    const double s2 = soft * soft;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        const double *r = src + 4 * (size_t)i;
        const int *ci = cc + 3 * (size_t)i;
        double e[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < n; ++j) {                 /* near: charges of the 27 cells around */
            if (j == i) continue;
            const int *cj = cc + 3 * (size_t)j;
            if (abs(cj[0] - ci[0]) > 1 || abs(cj[1] - ci[1]) > 1 || abs(cj[2] - ci[2]) > 1) continue;
            const double *q = src + 4 * (size_t)j;
            double d[3] = {r[0] - q[0], r[1] - q[1], r[2] - q[2]};
            double d2 = dot3(d, d) + s2;
            if (d2 == 0.0) continue;
            double w = q[3] / (d2 * sqrt(d2));
            for (int a = 0; a < 3; ++a) e[a] += w * d[a];
        }
        for (int c = 0; c < ncell; ++c) {             /* far: charge centres of the other cells */
            int cx = c % G, cy = (c / G) % G, cz = c / (G * G);
            if (abs(cx - ci[0]) <= 1 && abs(cy - ci[1]) <= 1 && abs(cz - ci[2]) <= 1) continue;
            for (int sg = 0; sg < 2; ++sg) {
                const double *ag = agg + (size_t)c * 8 + 4 * sg;
                if (ag[3] == 0.0) continue;
                double d[3] = {r[0] - ag[0], r[1] - ag[1], r[2] - ag[2]};
                double d2 = dot3(d, d) + s2;
                double w = ag[3] / (d2 * sqrt(d2));
                for (int a = 0; a < 3; ++a) e[a] += w * d[a];
            }
        }
        for (int a = 0; a < 3; ++a) E[3 * (size_t)i + a] = OR_KC * e[a];
    }
    (void)cell;
    free(cell); free(cc); free(agg);
}

/*
 * Dense BEM matrix, Eqs. (BEMpot), (BEMfld), (matrixBEM), row-major n x n.
 *   electrode (ed) rows:   A_ij = Q_ij = k_C phi_j(r_i)
 *   dielectric (dd) rows:  A_ij = W_ij = (er+ + er-)/2 delta_ij
 *                                 + (er+ - er-)/(4 pi) F_j(r_i).n_i   (j != i)
 * r_i, n_i are the centroid and normal of cell i; er-/er+ are the relative
 * permittivities on the negative / positive side of cell i.  For j == i the
 * integral term vanishes for a flat cell (r_i - r' is in the cell's plane).
 */
void or_assemble(int np, const double *tri, const int *kind, const double *er_minus,
                 const double *er_plus, double *A)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < np; ++i) {
        double c[3], n[3], area;
        or_tri_geometry(tri + 9 * (size_t)i, c, n, &area);
        for (int j = 0; j < np; ++j) {
            double phi, F[3];
            or_tri_integrals(tri + 9 * (size_t)j, c, &phi, F);
            double aij;
            if (kind[i] == 0) {
                aij = OR_KC * phi;
            } else if (i == j) {
                aij = 0.5 * (er_plus[i] + er_minus[i]);
            } else {
                aij = (er_plus[i] - er_minus[i]) / (4.0 * OR_PI) * dot3(F, n);
            }
            A[(size_t)i * np + j] = aij;
        }
    }
}

/* Gaussian elimination with partial pivoting, in place; solves A x = b, x
 * returned in b.  Returns 0, or -1 on an exactly singular pivot.  (Sec. 2.2:
 * the dense system (matrixBEM) is solved directly.) */
int or_solve_gepp(int n, double *A, double *b)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(A[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)p * n + j]; A[(size_t)p * n + j] = t;
            }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        double piv = A[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double f = A[(size_t)i * n + k] / piv;
            if (f == 0.0) continue;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * b[j];
        b[i] = s / A[(size_t)i * n + i];
    }
    return 0;
}

/*
 * Influence of point charges on the cells, Eqs. (potpart), (fldpart): the
 * cell-averaged potential and field of the charges,
 *   Vbar_i = k_C sum_p q_p phi_i(r_p) / A_i
 *   Ebar_i = k_C sum_p q_p int_Ci (r - r_p)/|r - r_p|^3 dA / A_i
 *          = -k_C sum_p q_p F_i(r_p) / A_i
 * and the right-hand-side correction of Eqs. (BEMpotpart), (BEMfldpart):
 *   ed rows: -Vbar_i;   dd rows: -(er+ - er-) eps0 Ebar_i . n_i
 */
void or_influence_rhs(int np, const double *tri, const int *kind, const double *er_minus,
                      const double *er_plus, int nq, const double *src, double *drhs)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < np; ++i) {
        double c[3], n[3], area;
        or_tri_geometry(tri + 9 * (size_t)i, c, n, &area);
        double vs = 0.0, es[3] = {0, 0, 0};
        for (int p = 0; p < nq; ++p) {
            double phi, F[3];
            or_tri_integrals(tri + 9 * (size_t)i, src + 4 * (size_t)p, &phi, F);
            double q = src[4 * (size_t)p + 3];
            vs += q * phi;
            es[0] -= q * F[0]; es[1] -= q * F[1]; es[2] -= q * F[2];
        }
        if (kind[i] == 0) drhs[i] = -OR_KC * vs / area;
        else drhs[i] = -(er_plus[i] - er_minus[i]) * OR_EPS0 * OR_KC * dot3(es, n) / area;
    }
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter-based RNG.      */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* The tracking step, IEEE binary32, one rounding per operation.              */
/* ------------------------------------------------------------------------- */
enum { K_ELASTIC = 0, K_EXCITATION = 1, K_IONISATION = 2, K_ATTACHMENT = 3 };
enum { SP_ELECTRON = 0, SP_CATION = 1, SP_ANION = 2 };
enum { ST_OK = 0, ST_CAPACITY = -6, ST_TRIALS = -8 };

/* uniform in [0,1) from the top 24 bits of a 32-bit draw */
static float u01(uint32_t u) { return (float)(u >> 8) * 5.9604645e-08f; }

/* -ln(U) for U = ((u >> 8) + 1) 2^-24 in (0, 1]; written with basic binary32
 * operations only: U = 2^(e-24) f, f in [1,2), ln f = 2 atanh((f-1)/(f+1)) by
 * its odd series to t^13 (|t| < 1/3, truncation < 1e-8). */
static float neg_log_u(uint32_t u)
{
    uint32_t m = (u >> 8) + 1u;          /* 1 .. 2^24 */
    int e = 31 - __builtin_clz(m);       /* floor(log2 m) */
    float mf = (float)m;
    float f = mf / (float)(1u << e);     /* exact: power-of-two scaling */
    float t = (f - 1.0f) / (f + 1.0f);
    float t2 = t * t;
    float s = 0.07692308f;               /* 1/13 */
    s = s * t2 + 0.09090909f;            /* 1/11 */
    s = s * t2 + 0.11111111f;            /* 1/9  */
    s = s * t2 + 0.14285715f;            /* 1/7  */
    s = s * t2 + 0.2f;                   /* 1/5  */
    s = s * t2 + 0.33333334f;            /* 1/3  */
    s = s * t2 + 1.0f;
    float lnf = 2.0f * t * s;
    float a = (float)(24 - e) * 0.6931472f;
    return a - lnf;
}

/* sin and cos of a in [0, pi/2) by Taylor polynomials in a^2 (Horner),
 * binary32 basic operations only. */
static void sincos_q(float a, float *s, float *c)
{
    float a2 = a * a;
    float ps = -1.6059044e-10f;          /* -1/13! */
    ps = ps * a2 + 2.5052108e-08f;       /*  1/11! */
    ps = ps * a2 - 2.7557319e-06f;       /* -1/9!  */
    ps = ps * a2 + 0.0001984127f;        /*  1/7!  (sign applied below) */
    ps = ps * a2 - 0.008333334f;
    ps = ps * a2 + 0.16666667f;
    ps = ps * a2 - 1.0f;
    *s = -(a * ps);
    float pc = 2.0876756e-09f;           /*  1/12! */
    pc = pc * a2 - 2.755732e-07f;        /* -1/10! */
    pc = pc * a2 + 2.4801588e-05f;       /*  1/8!  */
    pc = pc * a2 - 0.0013888889f;        /* -1/6!  */
    pc = pc * a2 + 0.041666668f;         /*  1/4!  */
    pc = pc * a2 - 0.5f;
    pc = pc * a2 + 1.0f;
    *c = pc;
}

/* Isotropic unit direction from two 32-bit draws: cos(theta) = 1 - 2u,
 * phi = 2 pi u' with the quadrant from the top two of u''s 24 bits. */
static void iso_dir(uint32_t ua, uint32_t ub, float *d)
{
    float c = 1.0f - 2.0f * u01(ua);
    float cc = c * c;
    float om = 1.0f - cc;
    if (om < 0.0f) om = 0.0f;
    float s = sqrtf(om);
    uint32_t b = ub >> 8;
    uint32_t q = b >> 22;
    float f = (float)(b & 0x3FFFFFu) * 5.9604645e-08f;   /* [0, 1/4) */
    float a = f * 6.2831855f;
    float sa, ca;
    sincos_q(a, &sa, &ca);
    float cp, sp;
    if (q == 0) { cp = ca; sp = sa; }
    else if (q == 1) { cp = -sa; sp = ca; }
    else if (q == 2) { cp = -ca; sp = -sa; }
    else { cp = sa; sp = -ca; }
    d[0] = s * cp; d[1] = s * sp; d[2] = c;
}

/* one unit in the last place of x toward +inf (dir > 0) or -inf (dir < 0) */
static float ulp_step(float x, float dir)
{
    return nextafterf(x, dir > 0.0f ? INFINITY : -INFINITY);
}

typedef struct {
    /* primary parameters */
    double dt, T, N, M_amu, nu_ion, z_lo, z_hi, beta;
    uint32_t seed_lo, seed_hi;
    int trial_cap;
    /* gas table */
    int n_proc, n_e;
    const float *egrid, *xs, *thr, *nuc;
    const int *pkind, *pmode;
    /* derived binary32 constants */
    float dt_f, nu_max_e, nu_ion_f, half_nu_ion, E_therm, v_th_ion, qm[3], K_e, K_ion,
          two_m_over_M, KCE, N_f, z_lo_f, z_hi_f, rc2, ion_thr;
    int recomb_on;
    int coll_mode;     /* 0: null-collision trials; 1: the paper's per-step probability */
    /* cells that absorb charges crossing them (charging-up): binary32
     * vertices [ntri][9]; hit_on = 0: only the planes z_lo / z_hi absorb */
    int hit_on, ntri;
    const float *tri9;
} or_gas;

/* Derived constants: each is computed in FP64 from the primary parameters and
 * rounded once to binary32. */
static void gas_derive(or_gas *g)
{
    double M = g->M_amu > 0 ? g->M_amu * OR_AMU : INFINITY;
    g->dt_f = (float)g->dt;
    g->nu_ion_f = (float)g->nu_ion;
    g->half_nu_ion = (float)(0.5 * g->nu_ion);
    g->E_therm = (float)(1.5 * OR_KB * g->T / OR_E);
    g->v_th_ion = isinf(M) ? 0.0f : (float)sqrt(3.0 * OR_KB * g->T / M);
    g->qm[SP_ELECTRON] = (float)(-OR_E / OR_ME);
    g->qm[SP_CATION] = isinf(M) ? 0.0f : (float)(OR_E / M);
    g->qm[SP_ANION] = isinf(M) ? 0.0f : (float)(-OR_E / M);
    g->K_e = (float)(0.5 * OR_ME / OR_E);
    g->K_ion = isinf(M) ? 0.0f : (float)(0.5 * M / OR_E);
    g->two_m_over_M = isinf(M) ? 0.0f : (float)(2.0 * OR_ME / M);
    g->KCE = (float)(OR_KC * OR_E);
    g->N_f = (float)g->N;
    g->z_lo_f = (float)g->z_lo;
    g->z_hi_f = (float)g->z_hi;
    /* majorant of the electron collision frequency (null-collision method,
     * Skullerud 1968, cited in Sec. 3.3.1): constant-frequency processes add
     * their frequency; tabulated ones are bounded on every grid segment by
     * N max(sigma_tot(E_i), sigma_tot(E_i+1)) v(E_i+1). */
    double nuc = 0.0, best = 0.0;
    g->ion_thr = 0.0f;
    for (int j = 0; j < g->n_proc; ++j) {
        if (g->pmode[j] == 1) nuc += (double)g->nuc[j];
        if (g->pkind[j] == K_IONISATION && g->ion_thr == 0.0f) g->ion_thr = g->thr[j];
    }
    for (int i = 0; i + 1 < g->n_e; ++i) {
        double s0 = 0.0, s1 = 0.0;
        for (int j = 0; j < g->n_proc; ++j) {
            if (g->pmode[j] != 0) continue;
            s0 += (double)g->xs[(size_t)j * g->n_e + i];
            s1 += (double)g->xs[(size_t)j * g->n_e + i + 1];
        }
        double v1 = sqrt(2.0 * (double)g->egrid[i + 1] * OR_E / OR_ME);
        double b = g->N * (s0 > s1 ? s0 : s1) * v1;
        if (b > best) best = b;
    }
    g->nu_max_e = (float)(nuc + best);
    /* recombination capture radius: with a rate coefficient beta the sphere
     * swept in one step, R_c = (3 beta dt / 4 pi)^(1/3); with beta == 0 the
     * Coulomb distance of Eq. (distRecomb), k_C e / (2 E_ioni); beta < 0: off. */
    g->recomb_on = g->beta >= 0.0;
    double rc = 0.0;
    if (g->beta > 0.0) rc = cbrt(3.0 * g->beta * g->dt / (4.0 * OR_PI));
    else if (g->beta == 0.0 && g->ion_thr > 0.0f) rc = OR_KC * OR_E / (2.0 * (double)g->ion_thr);
    else if (g->beta == 0.0) g->recomb_on = 0;
    g->rc2 = (float)(rc * rc);
}

void or_gas_constants(const double *prm, int n_proc, int n_e, const float *egrid,
                      const float *xs, const int *pkind, const int *pmode, const float *thr,
                      const float *nuc, float *out)
{
    or_gas g;
    memset(&g, 0, sizeof g);
    g.dt = prm[0]; g.T = prm[1]; g.N = prm[2]; g.M_amu = prm[3]; g.nu_ion = prm[4];
    g.z_lo = prm[5]; g.z_hi = prm[6]; g.beta = prm[7];
    g.n_proc = n_proc; g.n_e = n_e; g.egrid = egrid; g.xs = xs; g.pkind = pkind; g.pmode = pmode;
    g.thr = thr; g.nuc = nuc;
    gas_derive(&g);
    out[0] = g.nu_max_e; out[1] = g.E_therm; out[2] = g.v_th_ion; out[3] = g.rc2;
    out[4] = g.KCE; out[5] = g.K_e; out[6] = g.two_m_over_M; out[7] = (float)g.recomb_on;
}

typedef struct {
    int n_out_sp;      /* spawn records written */
    int dead;          /* absorbed */
    int attached;
    int collisions;
    int trials;
    int status;
    int hit_cell;      /* cell that absorbed the charge, or -1 */
} flight_result;

typedef struct { float p[3], v[3]; float pi[3], vi[3]; uint32_t parent; } spawn_rec;

/* First cell crossed by the straight segment a -> b (the chord of one
 * ballistic sub-flight), by the Moller-Trumbore ray-triangle test evaluated
 * in binary32 with this operation order (the decision is shared with the GPU
 * bit for bit): edges e1 = v1 - v0, e2 = v2 - v0, d = b - a, h = d x e2,
 * det = e1.h (0: parallel, no hit), s = a - v0, u = (s.h)/det in [0, 1],
 * q = s x e1, v = (d.q)/det >= 0 with u + v <= 1, t = (e2.q)/det in [0, 1].
 * The smallest t wins, ties to the lower cell index.  Returns the cell or -1. */
static int seg_hit(const or_gas *g, const float *a, const float *b)
{
    int best = -1;
    float bt = 0.0f;
    const float d0 = b[0] - a[0], d1 = b[1] - a[1], d2 = b[2] - a[2];
    for (int k = 0; k < g->ntri; ++k) {
        const float *v = g->tri9 + 9 * (size_t)k;
        const float e10 = v[3] - v[0], e11 = v[4] - v[1], e12 = v[5] - v[2];
        const float e20 = v[6] - v[0], e21 = v[7] - v[1], e22 = v[8] - v[2];
        const float h0 = d1 * e22 - d2 * e21, h1 = d2 * e20 - d0 * e22, h2 = d0 * e21 - d1 * e20;
        const float det = e10 * h0 + e11 * h1 + e12 * h2;
        if (det == 0.0f) continue;
        const float inv = 1.0f / det;
        const float s0 = a[0] - v[0], s1 = a[1] - v[1], s2 = a[2] - v[2];
        const float u = (s0 * h0 + s1 * h1 + s2 * h2) * inv;
        if (!(u >= 0.0f && u <= 1.0f)) continue;
        const float q0 = s1 * e12 - s2 * e11, q1 = s2 * e10 - s0 * e12, q2 = s0 * e11 - s1 * e10;
        const float w = (d0 * q0 + d1 * q1 + d2 * q2) * inv;
        if (!(w >= 0.0f && u + w <= 1.0f)) continue;
        const float t = (e20 * q0 + e21 * q1 + e22 * q2) * inv;
        if (!(t >= 0.0f && t <= 1.0f)) continue;
        if (best < 0 || t < bt) { best = k; bt = t; }
    }
    return best;
}

/* Collision frequency of process j for an electron of energy eps and speed
 * (linear interpolation in energy on the float grid, zero below threshold). */
static float nu_proc(const or_gas *g, int j, float eps, float speed, int lo, float w)
{
    if (g->pmode[j] == 1) return g->nuc[j];
    float Ns = g->N_f * speed;
    float s0 = g->xs[(size_t)j * g->n_e + lo];
    float s1 = g->xs[(size_t)j * g->n_e + lo + 1];
    float ds = s1 - s0;
    float sg = s0 + w * ds;
    if (eps < g->thr[j]) sg = 0.0f;
    return Ns * sg;
}

/* grid segment and interpolation weight of energy eps */
static void egrid_locate(const or_gas *g, float eps, int *lo_out, float *w_out)
{
    int lo = 0, hi = g->n_e - 1;
    float w;
    if (eps < g->egrid[0]) { lo = 0; w = 0.0f; }
    else if (eps >= g->egrid[g->n_e - 1]) { lo = g->n_e - 2; w = 1.0f; }
    else {
        while (hi - lo > 1) { int mid = (lo + hi) / 2; if (g->egrid[mid] <= eps) lo = mid; else hi = mid; }
        w = (eps - g->egrid[lo]) / (g->egrid[lo + 1] - g->egrid[lo]);
    }
    *lo_out = lo;
    *w_out = w;
}

/* One collision trial of the charge at its current state (Sec. 3.3.1-3.3.3):
 * with x uniform in [0, scale), process j is taken when x < nu_1 + ... + nu_j
 * (none: a null collision).  Returns 0 when nothing happened (null, or an
 * ionisation without the energy for it), 1 after a collision, 2 when the
 * flight ends (attachment, or the spawn records are full: fr->status). */
static int collide(const or_gas *g, uint32_t id, uint32_t step, uint32_t k, const uint32_t *r, float x,
                   float *p, float *v, uint8_t *sp, spawn_rec *recs, int rec_cap, flight_result *fr)
{
    uint32_t key[2] = {g->seed_lo, g->seed_hi};
    float v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    float speed = sqrtf(v2);
    float d[3];
    if (*sp == SP_ELECTRON) {
        float eps = g->K_e * v2;
        int lo;
        float w;
        egrid_locate(g, eps, &lo, &w);
        float cum = 0.0f;
        int proc = -1;
        for (int j = 0; j < g->n_proc; ++j) {
            cum = cum + nu_proc(g, j, eps, speed, lo, w);
            if (x < cum) { proc = j; break; }
        }
        if (proc < 0) return 0;                     /* null collision */
        int kind = g->pkind[proc];
        if (kind == K_ELASTIC) {
            iso_dir(r[2], r[3], d);
            float cosx = 0.0f;
            if (speed > 0.0f) cosx = (v[0] * d[0] + v[1] * d[1] + v[2] * d[2]) / speed;
            float om = 1.0f - cosx;
            float loss = g->two_m_over_M * om;
            float f = 1.0f - loss;
            float sn = speed * sqrtf(f);
            v[0] = sn * d[0]; v[1] = sn * d[1]; v[2] = sn * d[2];
            fr->collisions += 1;
        } else if (kind == K_EXCITATION) {
            float e2 = eps - g->thr[proc];
            if (e2 < 0.0f) e2 = 0.0f;
            float sn = sqrtf(e2 / g->K_e);
            iso_dir(r[2], r[3], d);
            v[0] = sn * d[0]; v[1] = sn * d[1]; v[2] = sn * d[2];
            fr->collisions += 1;
        } else if (kind == K_IONISATION) {
            float er = eps - g->thr[proc];
            er = er - g->E_therm;
            if (!(er > 0.0f)) return 0;             /* not enough energy: null */
            if (fr->n_out_sp >= rec_cap) { fr->status = ST_CAPACITY; return 2; }
            float half = 0.5f * er;
            float sn = sqrtf(half / g->K_e);
            iso_dir(r[2], r[3], d);
            float rr = g->KCE / (2.0f * er);
            float o[3] = {rr * d[0], rr * d[1], rr * d[2]};
            spawn_rec *sr = &recs[fr->n_out_sp];
            float pn[3], pp[3];
            for (int c = 0; c < 3; ++c) { pn[c] = p[c] + o[c]; pp[c] = p[c] - o[c]; }
            if (pn[0] == p[0] && pn[1] == p[1] && pn[2] == p[2]) {
                int ax = 0;
                float ad0 = fabsf(d[0]), ad1 = fabsf(d[1]), ad2 = fabsf(d[2]);
                if (ad1 > ad0) ax = 1;
                if (ad2 > (ax == 1 ? ad1 : ad0)) ax = 2;
                pn[ax] = ulp_step(p[ax], d[ax]);
                pp[ax] = ulp_step(p[ax], -d[ax]);
            }
            uint32_t ctr[4] = {id, step, k, 1u};
            uint32_t r2[4];
            or_philox4x32_10(ctr, key, r2);
            float di[3];
            iso_dir(r2[0], r2[1], di);
            for (int c = 0; c < 3; ++c) {
                sr->pi[c] = p[c];
                sr->vi[c] = g->v_th_ion * di[c];
                sr->p[c] = pn[c];
                sr->v[c] = sn * d[c];
                p[c] = pp[c];
                v[c] = -sn * d[c];
            }
            fr->n_out_sp += 1;
            fr->collisions += 1;
        } else { /* K_ATTACHMENT: the electron becomes an anion in place */
            iso_dir(r[2], r[3], d);
            for (int c = 0; c < 3; ++c) v[c] = g->v_th_ion * d[c];
            *sp = SP_ANION;
            fr->attached = 1;
            fr->collisions += 1;
            return 2;
        }
    } else {
        /* ions: constant frequency, half isotropic elastic (speed kept),
         * half charge exchange (fresh thermal velocity) */
        iso_dir(r[2], r[3], d);
        float sn = (x < g->half_nu_ion) ? speed : g->v_th_ion;
        v[0] = sn * d[0]; v[1] = sn * d[1]; v[2] = sn * d[2];
        fr->collisions += 1;
    }
    return 1;
}

/* Ballistic flight under the constant acceleration a for time fl (Sec. 3.2.5
 * Euler stepper: the field of the step start), then the absorbing planes. */
static int flight(const or_gas *g, float *p, float *v, const float *a, const float *ha, float fl)
{
    for (int c = 0; c < 3; ++c) {
        float w = ha[c] * fl;
        float x = v[c] + w;
        float y = x * fl;
        p[c] = p[c] + y;
        float dv = a[c] * fl;
        v[c] = v[c] + dv;
    }
    return p[2] <= g->z_lo_f || p[2] >= g->z_hi_f;
}

/*
 * Flight and collisions of one charge over one step dt under the step-start
 * field E (Sec. 3.2.5 Euler stepper: one field evaluation per step).  The
 * charge's state (p, v, species) is updated in place; ionisations append
 * spawn records (Sec. 3.3.3, Eq. (distIoni)).  A charge is absorbed where
 * the chord of a sub-flight crosses a cell (when cells absorb: charging-up,
 * Sec. 3.2.3) or where it ends beyond a plane z_lo / z_hi.  Collision
 * sampling:
 *   coll_mode 0 -- exact null-collision trials (Skullerud 1968, cited in
 *     Sec. 3.3.1): exponential waiting times -ln(U)/nu_max, process j taken
 *     with probability nu_j(eps)/nu_max at each trial;
 *   coll_mode 1 -- the paper's own scheme (Sec. 3.3.1): flight over the whole
 *     step, then one interaction with probability 1 - exp(-nu_tot(eps) dt),
 *     i.e. when -ln(U) < nu_tot dt, of type j with probability nu_j/nu_tot.
 */
static void fly_one(const or_gas *g, uint32_t id, uint32_t step, float *p, float *v,
                    uint8_t *sp, const float *E, spawn_rec *recs, int rec_cap,
                    flight_result *fr)
{
    uint32_t key[2] = {g->seed_lo, g->seed_hi};
    int s = *sp;
    float qm = g->qm[s];
    float a[3] = {qm * E[0], qm * E[1], qm * E[2]};
    float ha[3] = {0.5f * a[0], 0.5f * a[1], 0.5f * a[2]};
    if (g->coll_mode == 1) {
        const float p0[3] = {p[0], p[1], p[2]};
        const int crossed = flight(g, p, v, a, ha, g->dt_f);
        if (g->hit_on && (fr->hit_cell = seg_hit(g, p0, p)) >= 0) { fr->dead = 1; return; }
        if (crossed) { fr->dead = 1; return; }
        uint32_t ctr[4] = {id, step, 1u, 0u};
        uint32_t r[4];
        or_philox4x32_10(ctr, key, r);
        fr->trials += 1;
        float nu_tot;
        if (s == SP_ELECTRON) {
            float v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            float speed = sqrtf(v2);
            float eps = g->K_e * v2;
            int lo;
            float w;
            egrid_locate(g, eps, &lo, &w);
            nu_tot = 0.0f;
            for (int j = 0; j < g->n_proc; ++j) nu_tot = nu_tot + nu_proc(g, j, eps, speed, lo, w);
        } else {
            nu_tot = g->nu_ion_f;
        }
        float pr = nu_tot * g->dt_f;
        if (!(neg_log_u(r[0]) < pr)) return;        /* no interaction in this step */
        collide(g, id, step, 1u, r, u01(r[1]) * nu_tot, p, v, sp, recs, rec_cap, fr);
        return;
    }
    float numax = (s == SP_ELECTRON) ? g->nu_max_e : g->nu_ion_f;
    float t = 0.0f;
    uint32_t k = 0;
    for (;;) {
        float tau;
        uint32_t r[4] = {0, 0, 0, 0};
        if (numax > 0.0f) {
            k += 1;
            if ((int)k > g->trial_cap) { fr->status = ST_TRIALS; return; }
            uint32_t ctr[4] = {id, step, k, 0u};
            or_philox4x32_10(ctr, key, r);
            tau = neg_log_u(r[0]) / numax;
        } else {
            tau = INFINITY;
        }
        float tn = t + tau;
        float fl = (tn >= g->dt_f) ? (g->dt_f - t) : tau;
        const float p0[3] = {p[0], p[1], p[2]};
        const int crossed = flight(g, p, v, a, ha, fl);
        if (g->hit_on && (fr->hit_cell = seg_hit(g, p0, p)) >= 0) { fr->dead = 1; return; }
        if (crossed) { fr->dead = 1; return; }
        if (tn >= g->dt_f) return;
        t = tn;
        fr->trials += 1;
        if (collide(g, id, step, k, r, u01(r[1]) * numax, p, v, sp, recs, rec_cap, fr) == 2) return;
    }
}

/* Stats layout (doubles), shared by or_step's caller and the tests:
 *  0 n_before 1 n_after 2 n_e 3 n_cation 4 n_anion 5 spawned_pairs 6 absorbed
 *  7 attached 8 recombined_pairs 9 collisions 10 trials 11 required_capacity
 * 12..14 sum x,y,z (electrons) 15..17 sum x^2,y^2,z^2 (electrons)
 * 18..20 sum x,y,z (ions) 21..23 sum x^2,y^2,z^2 (ions) 24 sum kinetic energy of electrons (eV) */
#define OR_NSTATS 25
#define OR_MAX_TRIALS 256

/*
 * One tracking step of all charges (Sec. 3.2 - 3.3), in this order:
 *  1. (field at the step-start positions: E, given)
 *  2. recombination (Sec. 3.3.3, Eq. (distRecomb)): every electron proposes
 *     its nearest cation within R_c (binary32 squared distance, ties to the
 *     lower cation id; cations created in the previous step are exempt); every
 *     cation accepts the proposing electron with the smallest (d^2, id); both
 *     are removed;
 *  3. flight and collisions of the remaining charges (fly_one);
 *  4. compaction: survivors in their order, then the spawned charges ordered by
 *     (parent, trial, electron before cation), with new ids next_id, next_id+1..
 * Returns ST_OK, ST_CAPACITY (nothing written, stats[11] = required count) or
 * ST_TRIALS.
 */
int or_step(int n, const float *pos_q, const float *vel, const uint32_t *id,
            const uint32_t *birth, const uint8_t *species, const float *E,
            uint32_t step, uint32_t next_id, const double *prm,
            int n_proc, int n_e, const float *egrid, const float *xs, const int *pkind,
            const int *pmode, const float *thr, const float *nuc,
            int cap, float *o_pos_q, float *o_vel, uint32_t *o_id, uint32_t *o_birth,
            uint8_t *o_species, int *o_n, uint32_t *o_next_id, double *stats,
            int ntri, const float *tri9, int64_t *deposits)
{
    or_gas g;
    memset(&g, 0, sizeof g);
    g.dt = prm[0]; g.T = prm[1]; g.N = prm[2]; g.M_amu = prm[3]; g.nu_ion = prm[4];
    g.z_lo = prm[5]; g.z_hi = prm[6]; g.beta = prm[7];
    g.seed_lo = (uint32_t)prm[8]; g.seed_hi = (uint32_t)prm[9]; g.trial_cap = (int)prm[10];
    g.coll_mode = (int)prm[11];
    g.hit_on = prm[12] != 0.0 && ntri > 0;
    g.ntri = ntri;
    g.tri9 = tri9;
    g.n_proc = n_proc; g.n_e = n_e; g.egrid = egrid; g.xs = xs; g.pkind = pkind; g.pmode = pmode;
    g.thr = thr; g.nuc = nuc;
    gas_derive(&g);
    for (int i = 0; i < OR_NSTATS; ++i) stats[i] = 0.0;
    stats[0] = n;

    uint8_t *gone = calloc((size_t)n + 1, 1);
    /* 2. recombination */
    int recombined = 0;
    if (g.recomb_on) {
        int *prop = malloc(sizeof(int) * ((size_t)n + 1));
        float *pd2 = malloc(sizeof(float) * ((size_t)n + 1));
        for (int e = 0; e < n; ++e) {
            prop[e] = -1; pd2[e] = 0.0f;
            if (species[e] != SP_ELECTRON) continue;
            for (int c = 0; c < n; ++c) {
                if (species[c] != SP_CATION) continue;
                if (birth[c] != 0u && birth[c] == step) continue;
                float dx = pos_q[4 * e] - pos_q[4 * c];
                float dy = pos_q[4 * e + 1] - pos_q[4 * c + 1];
                float dz = pos_q[4 * e + 2] - pos_q[4 * c + 2];
                float d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 <= g.rc2)) continue;
                if (prop[e] < 0 || d2 < pd2[e] || (d2 == pd2[e] && id[c] < id[prop[e]])) {
                    prop[e] = c; pd2[e] = d2;
                }
            }
        }
        int *acc = malloc(sizeof(int) * ((size_t)n + 1));
        for (int c = 0; c < n; ++c) acc[c] = -1;
        for (int e = 0; e < n; ++e) {
            int c = prop[e];
            if (c < 0) continue;
            int b = acc[c];
            if (b < 0 || pd2[e] < pd2[b] || (pd2[e] == pd2[b] && id[e] < id[b])) acc[c] = e;
        }
        for (int c = 0; c < n; ++c)
            if (acc[c] >= 0) { gone[c] = 1; gone[acc[c]] = 1; recombined += 1; }
        free(prop); free(pd2); free(acc);
    }

    /* 3. flight */
    float *np_ = malloc(sizeof(float) * 4 * ((size_t)n + 1));
    float *nv_ = malloc(sizeof(float) * 4 * ((size_t)n + 1));
    uint8_t *nsp = malloc((size_t)n + 1);
    int rec_cap_total = 64;
    spawn_rec *recs = malloc(sizeof(spawn_rec) * rec_cap_total);
    int n_rec = 0;
    int status = ST_OK, absorbed = 0, attached = 0, collisions = 0, trials = 0;
    int *hit = malloc(sizeof(int) * ((size_t)n + 1));
    for (int i = 0; i < n; ++i) {
        hit[i] = -1;
        memcpy(np_ + 4 * (size_t)i, pos_q + 4 * (size_t)i, sizeof(float) * 4);
        memcpy(nv_ + 4 * (size_t)i, vel + 4 * (size_t)i, sizeof(float) * 4);
        nsp[i] = species[i];
        if (gone[i]) continue;
        spawn_rec local[OR_MAX_TRIALS];
        flight_result fr;
        memset(&fr, 0, sizeof fr);
        fr.hit_cell = -1;
        fly_one(&g, id[i], step, np_ + 4 * (size_t)i, nv_ + 4 * (size_t)i, &nsp[i],
                E + 3 * (size_t)i, local, OR_MAX_TRIALS, &fr);
        if (fr.status != ST_OK) { status = fr.status; break; }
        if (fr.dead) { gone[i] = 2; absorbed += 1; hit[i] = fr.hit_cell; }
        attached += fr.attached;
        collisions += fr.collisions;
        trials += fr.trials;
        for (int r = 0; r < fr.n_out_sp; ++r) {
            if (n_rec == rec_cap_total) {
                rec_cap_total *= 2;
                recs = realloc(recs, sizeof(spawn_rec) * rec_cap_total);
            }
            recs[n_rec] = local[r];
            recs[n_rec].parent = (uint32_t)i;
            n_rec += 1;
        }
    }
    int n_keep = 0;
    for (int i = 0; i < n; ++i) n_keep += gone[i] ? 0 : 1;
    int n_new = n_keep + 2 * n_rec;
    stats[5] = n_rec; stats[6] = absorbed; stats[7] = attached; stats[8] = recombined;
    stats[9] = collisions; stats[10] = trials; stats[11] = n_new;
    if (status == ST_OK && n_new > cap) status = ST_CAPACITY;
    if (status != ST_OK) {
        free(gone); free(np_); free(nv_); free(nsp); free(recs); free(hit);
        return status;
    }
    /* charges collected by cells (Eq. (charge-up) works with their sum per
     * cell), committed with the step */
    if (deposits)
        for (int i = 0; i < n; ++i)
            if (hit[i] >= 0) deposits[hit[i]] += pos_q[4 * (size_t)i + 3] > 0.0f ? 1 : -1;
    /* 4. compaction */
    int o = 0;
    for (int i = 0; i < n; ++i) {
        if (gone[i]) continue;
        memcpy(o_pos_q + 4 * (size_t)o, np_ + 4 * (size_t)i, sizeof(float) * 4);
        memcpy(o_vel + 4 * (size_t)o, nv_ + 4 * (size_t)i, sizeof(float) * 4);
        o_id[o] = id[i]; o_birth[o] = birth[i]; o_species[o] = nsp[i];
        o += 1;
    }
    uint32_t nid = next_id;
    for (int r = 0; r < n_rec; ++r) {
        spawn_rec *sr = &recs[r];
        for (int c = 0; c < 3; ++c) { o_pos_q[4 * (size_t)o + c] = sr->p[c]; o_vel[4 * (size_t)o + c] = sr->v[c]; }
        o_pos_q[4 * (size_t)o + 3] = -(float)OR_E; o_vel[4 * (size_t)o + 3] = 0.0f;
        o_id[o] = nid++; o_birth[o] = step + 1u; o_species[o] = SP_ELECTRON;
        o += 1;
        for (int c = 0; c < 3; ++c) { o_pos_q[4 * (size_t)o + c] = sr->pi[c]; o_vel[4 * (size_t)o + c] = sr->vi[c]; }
        o_pos_q[4 * (size_t)o + 3] = (float)OR_E; o_vel[4 * (size_t)o + 3] = 0.0f;
        o_id[o] = nid++; o_birth[o] = step + 1u; o_species[o] = SP_CATION;
        o += 1;
    }
    *o_n = o;
    *o_next_id = nid;
    stats[1] = o;
    for (int i = 0; i < o; ++i) {
        int s = o_species[i];
        const float *pp = o_pos_q + 4 * (size_t)i;
        if (s == SP_ELECTRON) {
            stats[2] += 1;
            for (int c = 0; c < 3; ++c) { stats[12 + c] += pp[c]; stats[15 + c] += (double)pp[c] * pp[c]; }
            const float *vv = o_vel + 4 * (size_t)i;
            double v2 = (double)vv[0] * vv[0] + (double)vv[1] * vv[1] + (double)vv[2] * vv[2];
            stats[24] += 0.5 * OR_ME * v2 / OR_E;
        } else {
            stats[s == SP_CATION ? 3 : 4] += 1;
            for (int c = 0; c < 3; ++c) { stats[18 + c] += pp[c]; stats[21 + c] += (double)pp[c] * pp[c]; }
        }
    }
    free(gone); free(np_); free(nv_); free(nsp); free(recs); free(hit);
    return ST_OK;
}

/* exported for the tests: the step's sampling helpers */
float or_neg_log_u(uint32_t u) { return neg_log_u(u); }
void or_iso_dir(uint32_t ua, uint32_t ub, float *d) { iso_dir(ua, ub, d); }
