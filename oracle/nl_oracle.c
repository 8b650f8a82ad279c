/*
 * CPU FP64 oracle for the nonlocal P1 tetrahedral assembly of
 * Chen, Ma & Zhang, "High performance implementation of 3D FEM for nonlocal
 * Poisson problem with different ball approximation strategies".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library and must be compiled with -ffp-contract=off.
 *
 * What it computes (plain, slow, in the paper's order):
 *   - the 4-point degree-2 Gauss rule on a tetrahedron (Sec. 4.3.1);
 *   - the element pairs (T, T') with T in Omega whose T' meets the ball
 *     B_delta(x_q) around some quadrature point x_q of T (Alg. 2 keeps the
 *     cells E with E cap B != empty);
 *   - per quadrature point, the approximate ball restricted to T'
 *     (Def. "simplex's dividing strategy", Def. "nocaps", Alg. 3; the
 *     simplified 3D approxcaps of Sec. 3.3; fullcaps = nocaps cells plus a
 *     Monte Carlo estimate over the cap region, Sec. 4.3.2 and Alg. 4;
 *     the element-level balls of Sec. 4.3: barycenter, overlap, inside,
 *     which take T' whole or not at all);
 *   - the local 8x8 contribution of Eqs. (notreplaced)/(replaceBasis):
 *     the integrand (phi_j(y)-phi_j(x))(phi_i(y)-phi_i(x)) psi evaluated at
 *     every inner quadrature point / accepted MC sample, with psi = gamma/2
 *     and the collar weight 2 of Eq. (Ah) for T' in the collar;
 *   - the load vector sum_T sum_q w_q phi_i(x_q) f (Alg. 5, last save).
 *
 * Readings of the paper used here (each is listed in the design notes):
 *   - psi = gamma/2, so that the operator int_B (u(y)-u(x)) gamma dy of
 *     |x|^2 is gamma*4*pi*delta^5/5 (= 6 for gamma = 15/(2 pi delta^5));
 *   - the Omega_I contribution uses the full difference form with weight 2,
 *     which for free nodes equals the paper's 2 phi_j phi_i int psi term and
 *     moves the volume constraint g (nodal) to the right-hand side;
 *   - a vertex is inside the open ball iff |v-x|^2 < delta^2;
 *   - the cap region for fullcaps is T' minus hull(I u P) (the paper's
 *     definition of the fullcap), split into the tetrahedra listed below;
 *   - Monte Carlo points come from Philox4x32-10 keyed by the seed with the
 *     counter (T, T', q, k).
 *
 * The few steps whose floating-point result decides an integer (vertex
 * classification, edge/sphere points, the m=2 diagonal, sub-tetrahedron
 * volumes for sampling, sample points and their acceptance) follow a fixed
 * operation order with no fused multiply-add, so that any implementation
 * following the same order takes the same decisions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "nl_oracle.h"

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Round: (hi0,lo0)=M0*c0, (hi1,lo1)=M1*c2,
 * c' = (hi1^c1^k0, lo1, hi0^c3^k1, lo0); the key is bumped by the Weyl
 * constants between rounds.                                                 */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* 4-point degree-2 rule (Sec. 4.3.1): barycentric (a,b,b,b) and its
 * permutations, a=(5+3 sqrt5)/20, b=(5-sqrt5)/20, weights |T|/4; a point
 * is b*(v0+v1+v2+v3) + (a-b)*v_q.                                           */
static const double QB  = 0x1.1b06d1d200913p-3;  /* (5-sqrt(5))/20   */
static const double QAB = 0x1.c9f25c5bfedd9p-2;  /* sqrt(5)/5 = a-b  */

static double det3(const double e1[3], const double e2[3], const double e3[3])
{
    return (e1[0] * (e2[1] * e3[2] - e2[2] * e3[1])
          + e1[1] * (e2[2] * e3[0] - e2[0] * e3[2]))
          + e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
}

static double orient4(const double p0[3], const double p1[3], const double p2[3], const double p3[3])
{
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) { e1[d] = p1[d] - p0[d]; e2[d] = p2[d] - p0[d]; e3[d] = p3[d] - p0[d]; }
    return det3(e1, e2, e3);
}

static double tet_volume(const double p0[3], const double p1[3], const double p2[3], const double p3[3])
{
    return fabs(orient4(p0, p1, p2, p3)) / 6.0;
}

double or_tet_volume(const double v[12])
{
    return tet_volume(v, v + 3, v + 6, v + 9);
}

void or_quad_points(const double v[12], double xq[12])
{
    for (int q = 0; q < 4; ++q)
        for (int d = 0; d < 3; ++d) {
            double s = (v[0 + d] + v[3 + d]) + (v[6 + d] + v[9 + d]);
            xq[3 * q + d] = QB * s + QAB * v[3 * q + d];
        }
}

/* Barycentric coordinates of y in the tetrahedron v (Cramer's rule). */
static void barycentric(const double v[4][3], const double y[3], double lam[4])
{
    double e1[3], e2[3], e3[3], r[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = v[1][d] - v[0][d]; e2[d] = v[2][d] - v[0][d]; e3[d] = v[3][d] - v[0][d];
        r[d] = y[d] - v[0][d];
    }
    double D = det3(e1, e2, e3);
    lam[1] = det3(r, e2, e3) / D;
    lam[2] = det3(e1, r, e3) / D;
    lam[3] = det3(e1, e2, r) / D;
    lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

/* ------------------------------------------------------------------------- */
/* Squared distance from p to the tetrahedron v: the closest point lies in
 * the relative interior of one face of the simplex (a vertex, an edge, a
 * triangle or the solid); enumerate them all, keep each unconstrained
 * projection that falls inside its face, and take the minimum.              */
static double sq(double a) { return a * a; }
static double dist2(const double a[3], const double b[3])
{
    return (sq(a[0] - b[0]) + sq(a[1] - b[1])) + sq(a[2] - b[2]);
}
static double dot3(const double a[3], const double b[3])
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

double or_dist2_point_tet(const double p[3], const double vflat[12])
{
    const double (*v)[3] = (const double (*)[3])vflat;
    double lam[4];
    barycentric(v, p, lam);
    if (lam[0] >= 0.0 && lam[1] >= 0.0 && lam[2] >= 0.0 && lam[3] >= 0.0) return 0.0;
    double best = INFINITY;
    for (int i = 0; i < 4; ++i) {
        double d = dist2(p, v[i]);
        if (d < best) best = d;
    }
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j) {
            double e[3], w[3];
            for (int d = 0; d < 3; ++d) { e[d] = v[j][d] - v[i][d]; w[d] = p[d] - v[i][d]; }
            double t = dot3(w, e) / dot3(e, e);
            if (t > 0.0 && t < 1.0) {
                double c[3];
                for (int d = 0; d < 3; ++d) c[d] = v[i][d] + t * e[d];
                double dd = dist2(p, c);
                if (dd < best) best = dd;
            }
        }
    for (int o = 0; o < 4; ++o) {
        int f[3], k = 0;
        for (int i = 0; i < 4; ++i) if (i != o) f[k++] = i;
        double e1[3], e2[3], w[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = v[f[1]][d] - v[f[0]][d];
            e2[d] = v[f[2]][d] - v[f[0]][d];
            w[d] = p[d] - v[f[0]][d];
        }
        double a11 = dot3(e1, e1), a12 = dot3(e1, e2), a22 = dot3(e2, e2);
        double b1 = dot3(e1, w), b2 = dot3(e2, w);
        double det = a11 * a22 - a12 * a12;
        double s = (b1 * a22 - b2 * a12) / det;
        double t = (a11 * b2 - a12 * b1) / det;
        if (s > 0.0 && t > 0.0 && s + t < 1.0) {
            double c[3];
            for (int d = 0; d < 3; ++d) c[d] = v[f[0]][d] + s * e1[d] + t * e2[d];
            double dd = dist2(p, c);
            if (dd < best) best = dd;
        }
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* Element pairs.  For every T in Omega (increasing id) list every T' with
 * min_q dist(x_q(T), T')^2 <= delta^2, sorted by T'.                        */
static void tet_coords(const double *verts, const int32_t *tets, int64_t t, double v[12])
{
    for (int k = 0; k < 4; ++k)
        for (int d = 0; d < 3; ++d) v[3 * k + d] = verts[3 * (int64_t)tets[4 * t + k] + d];
}

int or_pair_predicate(const double vT[12], const double vTp[12], double delta)
{
    double xq[12];
    or_quad_points(vT, xq);
    double d2 = delta * delta;
    for (int q = 0; q < 4; ++q)
        if (or_dist2_point_tet(xq + 3 * q, vTp) <= d2) return 1;
    return 0;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t or_pairs(const double *verts, int64_t nv, const int32_t *tets, int64_t nt,
                 const uint8_t *in_omega, double delta, int use_grid,
                 const int32_t *outer_list, int64_t n_list,
                 int64_t *ptr_out, int32_t *tp_out, int64_t cap)
{
    (void)nv;
    /* centroids and radii (max vertex distance from the centroid) */
    double *cen = (double *)malloc(sizeof(double) * 3 * (size_t)nt);
    double *rad = (double *)malloc(sizeof(double) * (size_t)nt);
    double rmax = 0.0, bmin[3] = {INFINITY, INFINITY, INFINITY}, bmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = 0; t < nt; ++t) {
        double v[12];
        tet_coords(verts, tets, t, v);
        for (int d = 0; d < 3; ++d) cen[3 * t + d] = 0.25 * ((v[d] + v[3 + d]) + (v[6 + d] + v[9 + d]));
        double r = 0.0;
        for (int k = 0; k < 4; ++k) { double dd = sqrt(dist2(v + 3 * k, cen + 3 * t)); if (dd > r) r = dd; }
        rad[t] = r; if (r > rmax) rmax = r;
        for (int d = 0; d < 3; ++d) { if (cen[3 * t + d] < bmin[d]) bmin[d] = cen[3 * t + d]; if (cen[3 * t + d] > bmax[d]) bmax[d] = cen[3 * t + d]; }
    }
    /* uniform grid of cell side >= delta + 2 rmax over the centroids */
    double cs = delta + 2.0 * rmax;
    int64_t gn[3];
    for (int d = 0; d < 3; ++d) { gn[d] = (int64_t)floor((bmax[d] - bmin[d]) / cs) + 1; if (gn[d] < 1) gn[d] = 1; }
    int64_t ncell = gn[0] * gn[1] * gn[2];
    int64_t *cstart = NULL, *cidx = NULL;
    int64_t *ccell = NULL;
    if (use_grid) {
        cstart = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
        cidx = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt);
        ccell = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt);
        for (int64_t t = 0; t < nt; ++t) {
            int64_t g[3];
            for (int d = 0; d < 3; ++d) {
                g[d] = (int64_t)floor((cen[3 * t + d] - bmin[d]) / cs);
                if (g[d] < 0) g[d] = 0;
                if (g[d] >= gn[d]) g[d] = gn[d] - 1;
            }
            ccell[t] = g[0] + gn[0] * (g[1] + gn[1] * g[2]);
            cstart[ccell[t] + 1]++;
        }
        for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
        memcpy(fill, cstart, sizeof(int64_t) * (size_t)ncell);
        for (int64_t t = 0; t < nt; ++t) cidx[fill[ccell[t]]++] = t;
        free(fill);
    }
    int64_t np = 0, nouter = 0;
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)nt);
    ptr_out[0] = 0;
    int64_t nloop = outer_list ? n_list : nt;
    for (int64_t li = 0; li < nloop; ++li) {
        int64_t t = outer_list ? (int64_t)outer_list[li] : li;
        if (!in_omega[t]) continue;
        double vT[12];
        tet_coords(verts, tets, t, vT);
        int64_t nb = 0;
        if (use_grid) {
            int64_t g[3] = {ccell[t] % gn[0], (ccell[t] / gn[0]) % gn[1], ccell[t] / (gn[0] * gn[1])};
            for (int64_t dz = -1; dz <= 1; ++dz)
                for (int64_t dy = -1; dy <= 1; ++dy)
                    for (int64_t dx = -1; dx <= 1; ++dx) {
                        int64_t x = g[0] + dx, y = g[1] + dy, z = g[2] + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= gn[0] || y >= gn[1] || z >= gn[2]) continue;
                        int64_t c = x + gn[0] * (y + gn[1] * z);
                        for (int64_t s = cstart[c]; s < cstart[c + 1]; ++s) {
                            int64_t tp = cidx[s];
                            double lim = (delta + rad[t] + rad[tp]) * (1.0 + 1e-9);
                            if (dist2(cen + 3 * t, cen + 3 * tp) > lim * lim) continue;
                            double vTp[12];
                            tet_coords(verts, tets, tp, vTp);
                            if (or_pair_predicate(vT, vTp, delta)) buf[nb++] = (int32_t)tp;
                        }
                    }
            qsort(buf, (size_t)nb, sizeof(int32_t), cmp_i32);
        } else {
            for (int64_t tp = 0; tp < nt; ++tp) {
                double vTp[12];
                tet_coords(verts, tets, tp, vTp);
                if (or_pair_predicate(vT, vTp, delta)) buf[nb++] = (int32_t)tp;
            }
        }
        if (tp_out && np + nb <= cap) memcpy(tp_out + np, buf, sizeof(int32_t) * (size_t)nb);
        np += nb;
        ptr_out[++nouter] = np;
    }
    free(buf); free(cen); free(rad);
    if (use_grid) { free(cstart); free(cidx); free(ccell); }
    return (np <= cap) ? np : -np;
}

/* ------------------------------------------------------------------------- */
/* Convex hull of a few points, split into tetrahedra by coning from the mean
 * point.  Brute force: every triple whose plane has all points on one side
 * spans a supporting plane; the points on that plane form one facet whose
 * 2D convex hull is fan-triangulated.                                       */
static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------- */
/* Exact sign of orientation determinants (Shewchuk, "Adaptive precision
 * floating-point arithmetic and fast robust geometric predicates", 1997):
 * a floating-point evaluation with an error bound, and, when the bound does
 * not decide, the exact value as a floating-point expansion (two_sum,
 * two_product with fma, expansion sums and scalings).                       */
#define EXP_MAX 512

static void two_sum(double a, double b, double *x, double *y)
{
    double s = a + b, bv = s - a, av = s - bv;
    *x = s;
    *y = (a - av) + (b - bv);
}

static void two_prod(double a, double b, double *x, double *y)
{
    double p = a * b;
    *x = p;
    *y = fma(a, b, -p);
}

/* h = e + f (nonoverlapping expansions, zero components dropped) */
static int exp_add(int elen, const double *e, int flen, const double *f, double *h)
{
    double tmp[EXP_MAX];
    int hlen = elen;
    for (int i = 0; i < elen; ++i) tmp[i] = e[i];
    for (int j = 0; j < flen; ++j) {
        double q = f[j];
        int k = 0;
        double out[EXP_MAX];
        for (int i = 0; i < hlen; ++i) {
            double x, y;
            two_sum(q, tmp[i], &x, &y);
            if (y != 0.0) out[k++] = y;
            q = x;
        }
        if (q != 0.0 || k == 0) out[k++] = q;
        for (int i = 0; i < k; ++i) tmp[i] = out[i];
        hlen = k;
    }
    for (int i = 0; i < hlen; ++i) h[i] = tmp[i];
    return hlen;
}

/* h = e * b */
static int exp_scale(int elen, const double *e, double b, double *h)
{
    double acc[EXP_MAX];
    int alen = 0;
    for (int i = 0; i < elen; ++i) {
        double p[2];
        two_prod(e[i], b, &p[1], &p[0]);
        alen = exp_add(alen, acc, 2, p, acc);
    }
    for (int i = 0; i < alen; ++i) h[i] = acc[i];
    return alen;
}

/* h = e * f */
static int exp_mul(int elen, const double *e, int flen, const double *f, double *h)
{
    double acc[EXP_MAX], t[EXP_MAX];
    int alen = 0;
    for (int j = 0; j < flen; ++j) {
        int tl = exp_scale(elen, e, f[j], t);
        alen = exp_add(alen, acc, tl, t, acc);
    }
    for (int i = 0; i < alen; ++i) h[i] = acc[i];
    return alen;
}

static int exp_sign(int n, const double *e)
{
    /* components are nonoverlapping and increasing in magnitude: the last
     * nonzero one carries the sign */
    for (int i = n - 1; i >= 0; --i) if (e[i] != 0.0) return e[i] > 0.0 ? 1 : -1;
    return 0;
}

/* sign of det[b-a; c-a; d-a] (the orientation of d against the plane abc) */
static int orient3d_sign(const double a[3], const double b[3], const double c[3], const double d[3])
{
    double u[3], v[3], w[3];
    for (int k = 0; k < 3; ++k) { u[k] = b[k] - a[k]; v[k] = c[k] - a[k]; w[k] = d[k] - a[k]; }
    double t0 = v[1] * w[2] - v[2] * w[1], t1 = v[2] * w[0] - v[0] * w[2], t2 = v[0] * w[1] - v[1] * w[0];
    double det = u[0] * t0 + u[1] * t1 + u[2] * t2;
    double perm = fabs(u[0]) * (fabs(v[1] * w[2]) + fabs(v[2] * w[1])) +
                  fabs(u[1]) * (fabs(v[2] * w[0]) + fabs(v[0] * w[2])) +
                  fabs(u[2]) * (fabs(v[0] * w[1]) + fabs(v[1] * w[0]));
    if (fabs(det) > 1e-14 * perm) return det > 0.0 ? 1 : -1;
    /* exact: differences as 2-component expansions, then the cofactor sum */
    double U[3][2], V[3][2], W[3][2];
    for (int k = 0; k < 3; ++k) {
        two_sum(b[k], -a[k], &U[k][1], &U[k][0]);
        two_sum(c[k], -a[k], &V[k][1], &V[k][0]);
        two_sum(d[k], -a[k], &W[k][1], &W[k][0]);
    }
    static const int cyc[3][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}};
    double total[EXP_MAX];
    int tl = 0;
    for (int r = 0; r < 3; ++r) {
        int i = cyc[r][0], j = cyc[r][1], k = cyc[r][2];
        double p1[EXP_MAX], p2[EXP_MAX], cf[EXP_MAX], term[EXP_MAX];
        int l1 = exp_mul(2, V[j], 2, W[k], p1);
        int l2 = exp_mul(2, V[k], 2, W[j], p2);
        for (int q = 0; q < l2; ++q) p2[q] = -p2[q];
        int lc = exp_add(l1, p1, l2, p2, cf);
        int lt = exp_mul(2, U[i], lc, cf, term);
        tl = exp_add(tl, total, lt, term, total);
    }
    return exp_sign(tl, total);
}

/* the triple is collinear iff its cross product is exactly zero */
static int collinear_exact(const double a[3], const double b[3], const double c[3])
{
    for (int k = 0; k < 3; ++k) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        /* 2D orientation in the (i,j) coordinate plane */
        double u0 = b[i] - a[i], u1 = b[j] - a[j], v0 = c[i] - a[i], v1 = c[j] - a[j];
        double det = u0 * v1 - u1 * v0;
        double perm = fabs(u0 * v1) + fabs(u1 * v0);
        if (fabs(det) > 1e-14 * perm) return 0;
        double U0[2], U1[2], V0[2], V1[2], p1[EXP_MAX], p2[EXP_MAX], tot[EXP_MAX];
        two_sum(b[i], -a[i], &U0[1], &U0[0]);
        two_sum(b[j], -a[j], &U1[1], &U1[0]);
        two_sum(c[i], -a[i], &V0[1], &V0[0]);
        two_sum(c[j], -a[j], &V1[1], &V1[0]);
        int l1 = exp_mul(2, U0, 2, V1, p1);
        int l2 = exp_mul(2, U1, 2, V0, p2);
        for (int q = 0; q < l2; ++q) p2[q] = -p2[q];
        int lt = exp_add(l1, p1, l2, p2, tot);
        if (exp_sign(lt, tot) != 0) return 0;
    }
    return 1;
}

/* 2D convex hull (monotone chain) of the points idx[0..m) projected on the
 * plane basis (u, w) through origin o; writes the polygon's point indices in
 * order and returns their number. */
static int polygon_2d(const double (*p)[3], const int *idx_in, int m, const double o[3], const double u[3],
                      const double w2[3], double ctol, int *poly)
{
    int idx[16];
    double px[16], py[16];
    for (int a = 0; a < m; ++a) {
        double r[3];
        for (int d = 0; d < 3; ++d) r[d] = p[idx_in[a]][d] - o[d];
        idx[a] = idx_in[a]; px[a] = dot3(r, u); py[a] = dot3(r, w2);
    }
    for (int a = 1; a < m; ++a) {             /* sort by (x, y) */
        int ti = idx[a]; double tx = px[a], ty = py[a]; int b = a - 1;
        while (b >= 0 && (px[b] > tx || (px[b] == tx && py[b] > ty))) {
            idx[b + 1] = idx[b]; px[b + 1] = px[b]; py[b + 1] = py[b]; b--;
        }
        idx[b + 1] = ti; px[b + 1] = tx; py[b + 1] = ty;
    }
    int hull[34], hn = 0;
    for (int a = 0; a < m; ++a) {             /* lower chain */
        while (hn >= 2) {
            int o2 = hull[hn - 2], b = hull[hn - 1];
            double cr = (px[b] - px[o2]) * (py[a] - py[o2]) - (py[b] - py[o2]) * (px[a] - px[o2]);
            if (cr <= ctol) hn--; else break;
        }
        hull[hn++] = a;
    }
    int lower = hn + 1;
    for (int a = m - 2; a >= 0; --a) {         /* upper chain */
        while (hn >= lower) {
            int o2 = hull[hn - 2], b = hull[hn - 1];
            double cr = (px[b] - px[o2]) * (py[a] - py[o2]) - (py[b] - py[o2]) * (px[a] - px[o2]);
            if (cr <= ctol) hn--; else break;
        }
        hull[hn++] = a;
    }
    hn--;                                      /* last point repeats the first */
    for (int a = 0; a < hn; ++a) poly[a] = idx[hull[a]];
    return hn < 0 ? 0 : hn;
}

/* Convex hull of a few points, split into tetrahedra coned from the mean
 * point.  `lab` (may be NULL) gives per point a bit set of known planes the
 * point lies on by construction (for the approximate ball: the faces of T');
 * a supporting plane through points sharing such a plane is that plane, with
 * exactly the points that carry its bit.  Other supporting planes are found
 * by brute force with exact orientation signs: every non-collinear triple
 * whose plane has all points on one side (points with a zero sign lie on
 * it).  The points of each facet are fan-triangulated along their 2D convex
 * hull. */
int or_hull_tets_labeled(int n, const double *pflat, const unsigned *lab, double *outflat, int maxout)
{
    const double (*p)[3] = (const double (*)[3])pflat;
    double (*out)[4][3] = (double (*)[4][3])outflat;
    if (n < 4 || n > 16) return 0;
    double c[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) for (int d = 0; d < 3; ++d) c[d] += p[i][d];
    for (int d = 0; d < 3; ++d) c[d] /= (double)n;
    double L = 0.0, Cabs = 0.0;
    for (int i = 0; i < n; ++i) {
        double dd = sqrt(dist2(p[i], c));
        if (dd > L) L = dd;
        for (int d = 0; d < 3; ++d) if (fabs(p[i][d]) > Cabs) Cabs = fabs(p[i][d]);
    }
    if (L == 0.0) return 0;
    (void)Cabs;
    uint32_t masks[600];
    int fi[600], nmask = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            for (int k = j + 1; k < n; ++k) {
                uint32_t mask = 0;
                unsigned shared = lab ? (lab[i] & lab[j] & lab[k]) : 0u;
                double e1[3], e2[3], nr[3];
                for (int d = 0; d < 3; ++d) { e1[d] = p[j][d] - p[i][d]; e2[d] = p[k][d] - p[i][d]; }
                cross3(e1, e2, nr);
                double nn = sqrt(dot3(nr, nr));
                if (shared) {
                    /* a known plane: its facet holds the points carrying that plane */
                    int bit = 0;
                    while (!(shared & (1u << bit))) bit++;
                    for (int l = 0; l < n; ++l) if (lab[l] & (1u << bit)) mask |= 1u << l;
                    if (nn <= 1e-14 * L * L) continue;        /* collinear triple */
                } else {
                    /* exact predicates: a collinear triple spans no plane */
                    if (collinear_exact(p[i], p[j], p[k])) continue;
                    int pos = 0, neg = 0;
                    for (int l = 0; l < n; ++l) {
                        int sg = (l == i || l == j || l == k) ? 0 : orient3d_sign(p[i], p[j], p[k], p[l]);
                        if (sg == 0) mask |= 1u << l;
                        else if (sg > 0) pos++;
                        else neg++;
                    }
                    if (pos && neg) continue;
                    if (!pos && !neg) return 0;                /* flat: zero volume */
                }
                int seen = 0;
                for (int m2 = 0; m2 < nmask; ++m2) if (masks[m2] == mask) { seen = 1; break; }
                if (seen || nmask >= 600) continue;
                masks[nmask] = mask;
                fi[nmask] = (i << 8) | (j << 4) | k;
                nmask++;
            }
    int nout = 0;
    for (int f = 0; f < nmask; ++f) {
        int sub = 0;
        for (int g = 0; g < nmask; ++g)
            if (g != f && (masks[f] & masks[g]) == masks[f] && masks[g] != masks[f]) { sub = 1; break; }
        if (sub) continue;
        uint32_t mask = masks[f];
        int i = fi[f] >> 8, j = (fi[f] >> 4) & 15, k = fi[f] & 15;
        double e1[3], e2[3], nr[3];
        for (int d = 0; d < 3; ++d) { e1[d] = p[j][d] - p[i][d]; e2[d] = p[k][d] - p[i][d]; }
        cross3(e1, e2, nr);
        double nn = sqrt(dot3(nr, nr));
        double u[3], w2[3], nh[3];
        for (int d = 0; d < 3; ++d) nh[d] = nr[d] / nn;
        double lu = sqrt(dot3(e1, e1));
        for (int d = 0; d < 3; ++d) u[d] = e1[d] / lu;
        cross3(nh, u, w2);
        int idx[16], m = 0, poly[16];
        for (int l = 0; l < n; ++l) if (mask & (1u << l)) idx[m++] = l;
        int hn = polygon_2d(p, idx, m, p[i], u, w2, 1e-14 * L * L, poly);
        for (int a = 1; a + 1 < hn; ++a) {
            if (nout >= maxout) return -1;
            const double *q0 = p[poly[0]], *q1 = p[poly[a]], *q2 = p[poly[a + 1]];
            for (int d = 0; d < 3; ++d) {
                out[nout][0][d] = c[d]; out[nout][1][d] = q0[d];
                out[nout][2][d] = q1[d]; out[nout][3][d] = q2[d];
            }
            nout++;
        }
    }
    return nout;
}

int or_hull_tets(int n, const double *pflat, double *outflat, int maxout)
{
    return or_hull_tets_labeled(n, pflat, NULL, outflat, maxout);
}

/* ------------------------------------------------------------------------- */
/* The approximate ball restricted to one element T' for the point x.        */

/* Intersection of the segment v_in -> v_out with the sphere |y-x| = delta. */
static void edge_sphere(const double vin[3], const double vout[3], const double x[3], double delta,
                        double p[3], double *tpar)
{
    double w[3], e[3];
    for (int d = 0; d < 3; ++d) { w[d] = vin[d] - x[d]; e[d] = vout[d] - vin[d]; }
    double A = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
    double B = (e[0] * w[0] + e[1] * w[1]) + e[2] * w[2];
    double C = ((w[0] * w[0] + w[1] * w[1]) + w[2] * w[2]) - delta * delta;
    double s = sqrt(B * B - A * C);
    double t = (B >= 0.0) ? (-C) / (B + s) : (s - B) / A;
    for (int d = 0; d < 3; ++d) p[d] = vin[d] + t * e[d];
    if (tpar) *tpar = t;
}

typedef struct {
    int m;                 /* number of vertices inside the open ball */
    int in[4], out[4];     /* local indices, ascending */
    double P[4][4][3];     /* P[i][o]: edge-sphere point between in-vertex i and out-vertex o */
} classify_t;

static void classify(const double v[4][3], const double x[3], double delta, classify_t *c)
{
    double d2 = delta * delta;
    int ni = 0, no = 0;
    for (int k = 0; k < 4; ++k) {
        double w[3];
        for (int d = 0; d < 3; ++d) w[d] = v[k][d] - x[d];
        double r2 = (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2];
        if (r2 < d2) c->in[ni++] = k; else c->out[no++] = k;
    }
    c->m = ni;
    for (int a = 0; a < ni; ++a)
        for (int b = 0; b < no; ++b)
            edge_sphere(v[c->in[a]], v[c->out[b]], x, delta, c->P[c->in[a]][c->out[b]], NULL);
}

/* Arc midpoints for approxcaps: for each face of T' crossed by the sphere
 * between two edge points p1,p2, the point of the circle (sphere cap plane)
 * on the far side of the chord p1p2 from the face's inside vertex, on the
 * perpendicular bisector of the chord; dropped if it is not in the face.   */
static int arc_midpoints(const double v[4][3], const double x[3], double delta, const classify_t *c,
                         double mu[4][3], int face[4])
{
    int inflag[4] = {0, 0, 0, 0};
    for (int a = 0; a < c->m; ++a) inflag[c->in[a]] = 1;
    int nm = 0;
    for (int o = 0; o < 4; ++o) {
        int f[3], k = 0;
        for (int i = 0; i < 4; ++i) if (i != o) f[k++] = i;
        const double *pp[2];
        int np = 0, vin = -1;
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b) {
                int i = f[a], j = f[b];
                if (inflag[i] && !inflag[j]) pp[np++] = c->P[i][j];
                else if (inflag[j] && !inflag[i]) pp[np++] = c->P[j][i];
            }
        for (int a = 0; a < 3; ++a) if (inflag[f[a]]) { vin = f[a]; break; }
        if (np != 2 || vin < 0) continue;
        double e1[3], e2[3], nr[3];
        for (int d = 0; d < 3; ++d) { e1[d] = v[f[1]][d] - v[f[0]][d]; e2[d] = v[f[2]][d] - v[f[0]][d]; }
        cross3(e1, e2, nr);
        double xw[3];
        for (int d = 0; d < 3; ++d) xw[d] = x[d] - v[f[0]][d];
        double s = dot3(xw, nr) / dot3(nr, nr);
        double cf[3];
        for (int d = 0; d < 3; ++d) cf[d] = x[d] - s * nr[d];
        double r2 = delta * delta - dist2(x, cf);
        if (!(r2 > 0.0)) continue;
        double mid[3], ch[3], w[3];
        for (int d = 0; d < 3; ++d) {
            mid[d] = 0.5 * (pp[0][d] + pp[1][d]);
            ch[d] = pp[1][d] - pp[0][d];
            w[d] = mid[d] - v[vin][d];
        }
        double cc = dot3(ch, ch);
        if (!(cc > 0.0)) continue;
        double pr = dot3(w, ch) / cc;
        for (int d = 0; d < 3; ++d) w[d] -= pr * ch[d];
        double lw = sqrt(dot3(w, w));
        if (!(lw > 0.0)) continue;
        double r = sqrt(r2);
        double m3[3];
        for (int d = 0; d < 3; ++d) m3[d] = cf[d] + r * (w[d] / lw);
        /* inside the face triangle? barycentric in the face plane */
        double g[3];
        for (int d = 0; d < 3; ++d) g[d] = m3[d] - v[f[0]][d];
        double a11 = dot3(e1, e1), a12 = dot3(e1, e2), a22 = dot3(e2, e2);
        double b1 = dot3(e1, g), b2 = dot3(e2, g);
        double det = a11 * a22 - a12 * a12;
        double ls = (b1 * a22 - b2 * a12) / det;
        double lt = (a11 * b2 - a12 * b1) / det;
        double tol = -1e-12;
        if (ls < tol || lt < tol || 1.0 - ls - lt < tol) continue;
        for (int d = 0; d < 3; ++d) mu[nm][d] = m3[d];
        face[nm] = o;
        nm++;
    }
    return nm;
}

/* Element-level approximate balls (Sec. 4.3: the element is taken whole or
 * not at all): barycenter - T' when its barycenter lies in the closed ball;
 * overlap - T' when it meets the closed ball; inside - T' when all four
 * vertices lie in the open ball.                                          */
static int element_level_full(const double v[4][3], const double x[3], double delta, int strategy,
                              const classify_t *c)
{
    const double d2 = delta * delta;
    if (strategy == OR_INSIDE) return c->m == 4;
    if (strategy == OR_OVERLAP) return or_dist2_point_tet(x, &v[0][0]) <= d2;
    double w[3];
    for (int d = 0; d < 3; ++d) w[d] = 0.25 * ((v[0][d] + v[1][d]) + (v[2][d] + v[3][d])) - x[d];
    return (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2] <= d2;
}

/* Deterministic cells of the approximate ball inside T' (nocaps/approxcaps,
 * the nocaps part of fullcaps, and T' itself or nothing for the
 * element-level strategies).  Returns the number of tetrahedra.            */
/* The cells of hull(I u P) (Def. simplexdiv: E_k^0, whose split into
 * simplices the paper leaves open; with a varying kernel the 4-point rule
 * depends on it): the cone from the first inside vertex a over the hull's
 * faces away from a, with the m = 2 diagonal of the cap table below.
 *   m = 1: (a, p_1, p_2, p_3), p_k the edge point towards the k-th outside
 *          vertex;
 *   m = 2: (a, b, c2, d2), then (a, c1, c2, d2) (a, c1, d2, d1), or with the
 *          diagonal c2-d1 (a, c1, c2, d1) (a, c2, d2, d1), where c1, d1 are
 *          the edge points from a and c2, d2 those from b (towards the
 *          first and second outside vertex);
 *   m = 3: (a, f1, f2, f3) (a, b, c, f3) (a, b, f3, f2), f_k the edge point
 *          from the k-th inside vertex.                                     */
static int nocaps_cells(const double v[4][3], const classify_t *c, double S[3][4][3]);

static int region_cells(const double v[4][3], const double x[3], double delta, int strategy,
                        const classify_t *c, double cells[][4][3], int maxcells)
{
    if (strategy >= OR_BARYCENTER) {
        if (!element_level_full(v, x, delta, strategy, c)) return 0;
        memcpy(cells[0], v, sizeof(double) * 12);
        return 1;
    }
    if (c->m == 4) {
        memcpy(cells[0], v, sizeof(double) * 12);
        return 1;
    }
    if (c->m == 0) return 0;
    if (strategy != OR_APPROXCAPS && maxcells >= 3) return nocaps_cells(v, c, (double (*)[4][3])cells);
    /* each point carries the faces of T' it lies on (face f = opposite vertex
     * f): a vertex k lies on the faces f != k, an edge point (i,o) on the
     * faces f not in {i,o}, an arc midpoint of face o on face o */
    double pts[16][3];
    unsigned lab[16];
    int n = 0;
    for (int a = 0; a < c->m; ++a) {
        lab[n] = 15u & ~(1u << c->in[a]);
        memcpy(pts[n++], v[c->in[a]], sizeof(double) * 3);
    }
    for (int a = 0; a < c->m; ++a)
        for (int b = 0; b < 4 - c->m; ++b) {
            lab[n] = 15u & ~((1u << c->in[a]) | (1u << c->out[b]));
            memcpy(pts[n++], c->P[c->in[a]][c->out[b]], sizeof(double) * 3);
        }
    if (strategy == OR_APPROXCAPS) {
        double mu[4][3];
        int face[4];
        int nm = arc_midpoints(v, x, delta, c, mu, face);
        for (int a = 0; a < nm; ++a) {
            lab[n] = 1u << face[a];
            memcpy(pts[n++], mu[a], sizeof(double) * 3);
        }
    }
    int k = or_hull_tets_labeled(n, &pts[0][0], lab, &cells[0][0][0], maxcells);
    return k < 0 ? 0 : k;
}

/* The cap region S = T' minus hull(I u P), as a fixed list of tetrahedra
 * (vertex order matters: sample points are built from it).
 *   m=0: (v0,v1,v2,v3).
 *   m=1: I={a}, O={b,c,d}, e_k = P(a,.): (b,e1,e2,e3), (b,c,d,e3), (b,c,e3,e2).
 *   m=2: I={a,b}, O={c,d}, c1=P(a,c), d1=P(a,d), c2=P(b,c), d2=P(b,d); the
 *        skew quad c1-c2-d2-d1 of hull(I u P) is split on the diagonal c1-d2
 *        unless orient(c1,c2,d2,d1) and orient(c1,c2,d2,a) have strictly
 *        opposite signs, then on c2-d1:
 *        c1-d2: (c,d,d1,d2), (c,c1,c2,d2), (c,c1,d2,d1);
 *        c2-d1: (c,d,d1,d2), (c,c1,c2,d1), (c,c2,d2,d1).
 *   m=3: I={a,b,c}, O={d}: (d, P(a,d), P(b,d), P(c,d)).                     */
static void cpy3(double d[3], const double s[3]) { d[0] = s[0]; d[1] = s[1]; d[2] = s[2]; }
static void set_tet(double t[4][3], const double *a, const double *b, const double *c, const double *d)
{
    cpy3(t[0], a); cpy3(t[1], b); cpy3(t[2], c); cpy3(t[3], d);
}

static int m2_other_diagonal(const double v[4][3], const classify_t *c)
{
    int a = c->in[0], cc = c->out[0], d = c->out[1], b = c->in[1];
    const double *c1 = c->P[a][cc], *d1 = c->P[a][d], *c2 = c->P[b][cc], *d2 = c->P[b][d];
    double o1 = orient4(c1, c2, d2, d1), o2 = orient4(c1, c2, d2, v[a]);
    return (o1 > 0.0 && o2 < 0.0) || (o1 < 0.0 && o2 > 0.0);
}

static int nocaps_cells(const double v[4][3], const classify_t *c, double S[3][4][3])
{
    switch (c->m) {
    case 1: {
        int a = c->in[0];
        set_tet(S[0], v[a], c->P[a][c->out[0]], c->P[a][c->out[1]], c->P[a][c->out[2]]);
        return 1;
    }
    case 2: {
        int a = c->in[0], b = c->in[1], cc = c->out[0], d = c->out[1];
        const double *c1 = c->P[a][cc], *d1 = c->P[a][d], *c2 = c->P[b][cc], *d2 = c->P[b][d];
        set_tet(S[0], v[a], v[b], c2, d2);
        if (!m2_other_diagonal(v, c)) { set_tet(S[1], v[a], c1, c2, d2); set_tet(S[2], v[a], c1, d2, d1); }
        else                          { set_tet(S[1], v[a], c1, c2, d1); set_tet(S[2], v[a], c2, d2, d1); }
        return 3;
    }
    case 3: {
        int a = c->in[0], b = c->in[1], cc = c->in[2], d = c->out[0];
        const double *f1 = c->P[a][d], *f2 = c->P[b][d], *f3 = c->P[cc][d];
        set_tet(S[0], v[a], f1, f2, f3);
        set_tet(S[1], v[a], v[b], v[cc], f3);
        set_tet(S[2], v[a], v[b], f3, f2);
        return 3;
    }
    default:
        return 0;
    }
}

static int cap_cells(const double v[4][3], const classify_t *c, double S[3][4][3])
{
    switch (c->m) {
    case 0:
        set_tet(S[0], v[0], v[1], v[2], v[3]);
        return 1;
    case 1: {
        int a = c->in[0], b = c->out[0], cc = c->out[1], d = c->out[2];
        const double *e1 = c->P[a][b], *e2 = c->P[a][cc], *e3 = c->P[a][d];
        set_tet(S[0], v[b], e1, e2, e3);
        set_tet(S[1], v[b], v[cc], v[d], e3);
        set_tet(S[2], v[b], v[cc], e3, e2);
        return 3;
    }
    case 2: {
        int a = c->in[0], b = c->in[1], cc = c->out[0], d = c->out[1];
        const double *c1 = c->P[a][cc], *d1 = c->P[a][d], *c2 = c->P[b][cc], *d2 = c->P[b][d];
        int other = m2_other_diagonal(v, c);
        set_tet(S[0], v[cc], v[d], d1, d2);
        if (!other) { set_tet(S[1], v[cc], c1, c2, d2); set_tet(S[2], v[cc], c1, d2, d1); }
        else        { set_tet(S[1], v[cc], c1, c2, d1); set_tet(S[2], v[cc], c2, d2, d1); }
        return 3;
    }
    case 3: {
        int a = c->in[0], b = c->in[1], cc = c->in[2], d = c->out[0];
        set_tet(S[0], v[d], c->P[a][d], c->P[b][d], c->P[cc][d]);
        return 1;
    }
    default:
        return 0;
    }
}

/* One Monte Carlo sample in the cap region: sub-tetrahedron chosen by
 * cumulative volume with u0, a uniform point in it from the sorted
 * uniforms u1..u3 (spacings of three ordered uniforms are uniform on the
 * simplex).                                                                 */
void or_mc_point(const double *Sflat, int ns, const uint32_t u[4], double y[3], int *which)
{
    const double (*S)[4][3] = (const double (*)[4][3])Sflat;
    double vol[3], tot = 0.0;
    for (int j = 0; j < ns; ++j) { vol[j] = tet_volume(S[j][0], S[j][1], S[j][2], S[j][3]); tot += vol[j]; }
    double r = ((double)u[0] * 0x1p-32) * tot;
    int j = ns - 1;
    double cum = 0.0;
    for (int k = 0; k < ns; ++k) { cum += vol[k]; if (r < cum) { j = k; break; } }
    double U[3];
    for (int k = 0; k < 3; ++k) U[k] = ((double)u[k + 1] + 0.5) * 0x1p-32;
    /* sort three values ascending */
    if (U[0] > U[1]) { double t = U[0]; U[0] = U[1]; U[1] = t; }
    if (U[1] > U[2]) { double t = U[1]; U[1] = U[2]; U[2] = t; }
    if (U[0] > U[1]) { double t = U[0]; U[0] = U[1]; U[1] = t; }
    double be[4] = {U[0], U[1] - U[0], U[2] - U[1], 1.0 - U[2]};
    for (int d = 0; d < 3; ++d)
        y[d] = ((be[0] * S[j][0][d] + be[1] * S[j][1][d]) + be[2] * S[j][2][d]) + be[3] * S[j][3][d];
    if (which) *which = j;
}

/* ------------------------------------------------------------------------- */
/* Sobol' points in four dimensions (Sobol' 1967), for the quasi-Monte Carlo
 * form of the cap integral.  The paper leaves better sampling over the caps
 * open (Sec. 4.3.2: uniform points often fall outside the fullcap); this is
 * one such choice, outside the paper's own method.
 * Direction numbers of dimension d, bit b (b = 0 the most significant):
 * v = m_{b+1} 2^(31-b), with m_k odd and m_k < 2^k.  Dimension 0 has
 * m_k = 1 for every k (the van der Corput sequence).  Dimensions 1..3 take
 * the primitive polynomials x + 1, x^2 + x + 1 and x^3 + x + 1 with the
 * initial values m = (1), (1, 3) and (1, 3, 1) of Joe & Kuo's table (2008),
 * and for k > s (s the degree, a_1 .. a_{s-1} the inner coefficients)
 *   m_k = 2 a_1 m_{k-1} ^ 4 a_2 m_{k-2} ^ ... ^ 2^s m_{k-s} ^ m_{k-s}.
 * Point k is the one of index g = k ^ (k >> 1) (Gray-code order, Antonov &
 * Saleev 1979): the XOR of the direction numbers of the bits set in g.     */
static void sobol_dirs(uint32_t v[4][32])
{
    static const int deg[4] = {0, 1, 2, 3};
    static const unsigned inner[4] = {0, 0, 1, 1};     /* a_1 .. a_{s-1}, a_1 the high bit */
    static const uint32_t init[4][3] = {{0, 0, 0}, {1, 0, 0}, {1, 3, 0}, {1, 3, 1}};
    for (int b = 0; b < 32; ++b) v[0][b] = 1u << (31 - b);
    for (int d = 1; d < 4; ++d) {
        const int s = deg[d];
        uint32_t m[33];
        for (int k = 1; k <= s; ++k) m[k] = init[d][k - 1];
        for (int k = s + 1; k <= 32; ++k) {
            uint32_t x = m[k - s] ^ (m[k - s] << s);
            for (int i = 1; i < s; ++i)
                if ((inner[d] >> (s - 1 - i)) & 1u) x ^= m[k - i] << i;
            m[k] = x;
        }
        for (int b = 0; b < 32; ++b) v[d][b] = m[b + 1] << (31 - b);
    }
}

void or_sobol_point(uint32_t k, uint32_t out[4])
{
    uint32_t v[4][32];
    sobol_dirs(v);
    const uint32_t g = k ^ (k >> 1);
    for (int d = 0; d < 4; ++d) {
        uint32_t x = 0;
        for (int b = 0; b < 32; ++b)
            if ((g >> b) & 1u) x ^= v[d][b];
        out[d] = x;
    }
}

/* Cube root of a > 0 by Newton's method, x <- x - (x^3 - a) / (3 x^2),
 * six steps from 2^q (1 + (m 2^r - 1)/3) where a = m 2^(3q + r),
 * m in [0.5, 1), r in {0, 1, 2}: the start is within 0.2 of the root's
 * mantissa, and six quadratic steps reach double precision.               */
static double cbrt_newton(double a)
{
    int e;
    double m = frexp(a, &e);
    int q = e / 3, r = e - 3 * q;
    if (r < 0) { r += 3; q -= 1; }
    double x = ldexp(1.0 + (ldexp(m, r) - 1.0) / 3.0, q);
    for (int i = 0; i < 6; ++i) x = x - (x * x * x - a) / (3.0 * (x * x));
    return x;
}

/* Quasi-Monte Carlo point: the cell from u[0] as for or_mc_point, and the
 * point in the cell by the nested map of the unit cube onto the simplex,
 * s = U1^(1/3), t = U2^(1/2), w = U3 (U_k the uniforms of u[k]):
 * beta = (1 - s, s (1 - t), s t (1 - w), s t w), which is uniform on the
 * cell and, unlike sorted uniforms, continuous in (U1, U2, U3), as
 * low-discrepancy points need.                                             */
void or_qmc_point(const double *Sflat, int ns, const uint32_t u[4], double y[3], int *which)
{
    const double (*S)[4][3] = (const double (*)[4][3])Sflat;
    double vol[3], tot = 0.0;
    for (int j = 0; j < ns; ++j) { vol[j] = tet_volume(S[j][0], S[j][1], S[j][2], S[j][3]); tot += vol[j]; }
    double r = ((double)u[0] * 0x1p-32) * tot;
    int j = ns - 1;
    double cum = 0.0;
    for (int k = 0; k < ns; ++k) { cum += vol[k]; if (r < cum) { j = k; break; } }
    double U[3];
    for (int k = 0; k < 3; ++k) U[k] = ((double)u[k + 1] + 0.5) * 0x1p-32;
    double s = cbrt_newton(U[0]), t = sqrt(U[1]), w = U[2];
    double st = s * t;
    double be[4] = {1.0 - s, s * (1.0 - t), st * (1.0 - w), st * w};
    for (int d = 0; d < 3; ++d)
        y[d] = ((be[0] * S[j][0][d] + be[1] * S[j][1][d]) + be[2] * S[j][2][d]) + be[3] * S[j][3][d];
    if (which) *which = j;
}

/* The Monte Carlo samples of the cap S = T' minus hull(I u P) around x
 * (Sec. 4.3.2, Alg. 4).  The cap exists only when T' meets the closed ball:
 * some vertex inside, or, with none inside, the distance from x to T' at
 * most delta.  Then nmc samples are drawn with key = seed and counter
 * (idT, idTp, q, k); each is handed to fn with its cap cell and whether
 * |y - x|^2 <= delta^2, together with the weight |S|/nmc.  Returns the number
 * of samples drawn (0 when there is no cap).                                */
typedef void (*sample_fn)(void *ctx, int k, const double y[3], int cell, int accepted, double wgt);

/* With qmc, sample k takes the words of Sobol' point k (or_sobol_point),
 * each XORed with a word of one Philox draw with counter (idT, idTp, q,
 * 0xFFFFFFFF) (a digital shift, which leaves every point uniform on the 2^32
 * grid and keeps the net structure), in place of the Philox draw of counter
 * (idT, idTp, q, k); the cell choice follows from the words as for Monte
 * Carlo, the point from the nested map of or_qmc_point.                     */
static int cap_samples(const double v[4][3], const double vTp[12], const double x[3], double delta,
                       const classify_t *c, int nmc, uint64_t seed, uint32_t idT, uint32_t idTp, uint32_t q,
                       int qmc, sample_fn fn, void *ctx)
{
    if (c->m == 4 || nmc <= 0) return 0;
    if (c->m == 0 && !(or_dist2_point_tet(x, vTp) <= delta * delta)) return 0;
    double S[3][4][3];
    int ns = cap_cells(v, c, S);
    double tot = 0.0;
    for (int j = 0; j < ns; ++j) tot += tet_volume(S[j][0], S[j][1], S[j][2], S[j][3]);
    double wgt = tot / (double)nmc;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double d2 = delta * delta;
    uint32_t shift[4] = {0, 0, 0, 0};
    if (qmc) {
        uint32_t ctr[4] = {idT, idTp, q, 0xFFFFFFFFu};
        or_philox4x32_10(ctr, key, shift);
    }
    for (int k = 0; k < nmc; ++k) {
        uint32_t u[4];
        if (qmc) {
            or_sobol_point((uint32_t)k, u);
            for (int d = 0; d < 4; ++d) u[d] ^= shift[d];
        } else {
            uint32_t ctr[4] = {idT, idTp, q, (uint32_t)k};
            or_philox4x32_10(ctr, key, u);
        }
        double y[3];
        int which = 0;
        if (qmc) or_qmc_point(&S[0][0][0], ns, u, y, &which);
        else or_mc_point(&S[0][0][0], ns, u, y, &which);
        double w[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
        double r2 = (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2];
        fn(ctx, k, y, which, r2 <= d2, wgt);
    }
    return nmc;
}

/* ------------------------------------------------------------------------- */
/* Moments of the approximate ball inside T' around x: M[0] = |R|,
 * M[1+a] = int_R lambda'_a, M[5..14] = int_R lambda'_a lambda'_b (a<=b,
 * row-major upper triangle), with lambda' the barycentric coordinates of T'.
 * Inner integrals use the 4-point rule on every cell (Sec. 4.3.1) and the
 * Monte Carlo estimate |S|/N sum 1{|y-x|<=delta} on the cap (Sec. 4.3.2).
 * Returns the number of accepted samples; *mc_vol receives the MC part of
 * M[0].                                                                     */
/* Kernel shape phi on the ball: the kernel is gamma phi(|x - y|) (Sec. 2,
 * with the constant kernel as phi = 1).  kpoly NULL: phi = 1; otherwise the
 * polynomial phi = c0 + c1 s + c2 s^2 + c3 s^3 in s = |x - y|^2 / delta^2,
 * kpoly = (c0, c1, c2, c3), with s capped at 1: the element-level strategies
 * take T' whole and so place points past the sphere, where phi keeps its
 * value on the sphere.  The inner integrals weight every point of the
 * 4-point rule and every accepted cap sample by phi there (Sec. 4.3.1 keeps
 * the 4-point rule, no longer exact when phi varies).                      */
static double kshape(const double *kpoly, const double x[3], const double y[3], double delta)
{
    if (!kpoly) return 1.0;
    double s = dist2(x, y) / (delta * delta);
    if (s > 1.0) s = 1.0;
    return kpoly[0] + s * (kpoly[1] + s * (kpoly[2] + s * kpoly[3]));
}

static void add_point(double M[15], const double v[4][3], const double y[3], double w)
{
    double lam[4];
    barycentric(v, y, lam);
    M[0] += w;
    for (int a = 0; a < 4; ++a) M[1 + a] += w * lam[a];
    int k = 5;
    for (int a = 0; a < 4; ++a)
        for (int b = a; b < 4; ++b) M[k++] += w * lam[a] * lam[b];
}

/* accepted samples add 1, lambda'(y) and lambda'(y) lambda'(y)^T times |S|/N */
struct moments_ctx {
    double *M;
    const double (*v)[3];
    int acc;
    double *mc_vol;
    const double *kpoly;
    const double *x;
    double delta;
};

static void moments_sample(void *p, int k, const double y[3], int cell, int accepted, double wgt)
{
    struct moments_ctx *ctx = (struct moments_ctx *)p;
    (void)k; (void)cell;
    if (!accepted) return;
    const double w = wgt * kshape(ctx->kpoly, ctx->x, y, ctx->delta);
    add_point(ctx->M, ctx->v, y, w);
    ctx->acc++;
    if (ctx->mc_vol) *ctx->mc_vol += w;
}

int or_region_moments(const double vTp[12], const double x[3], double delta, int strategy,
                      int nmc, uint64_t seed, uint32_t idT, uint32_t idTp, uint32_t q,
                      const double *kpoly, double M[15], double *mc_vol)
{
    const double (*v)[3] = (const double (*)[3])vTp;
    const int qmc = strategy == OR_FULLCAPS_QMC;
    if (qmc) strategy = OR_FULLCAPS;
    memset(M, 0, sizeof(double) * 15);
    if (mc_vol) *mc_vol = 0.0;
    classify_t c;
    classify(v, x, delta, &c);
    double cells[256][4][3];
    int nc = region_cells(v, x, delta, strategy, &c, cells, 256);
    for (int s = 0; s < nc; ++s) {
        double vol = tet_volume(cells[s][0], cells[s][1], cells[s][2], cells[s][3]);
        double flat[12], yq[12];
        memcpy(flat, cells[s], sizeof(flat));
        or_quad_points(flat, yq);
        for (int k = 0; k < 4; ++k) add_point(M, v, yq + 3 * k, (vol / 4.0) * kshape(kpoly, x, yq + 3 * k, delta));
    }
    struct moments_ctx mc = {M, v, 0, mc_vol, kpoly, x, delta};
    if (strategy == OR_FULLCAPS)
        cap_samples(v, vTp, x, delta, &c, nmc, seed, idT, idTp, q, qmc, moments_sample, &mc);
    return mc.acc;
}

/* ------------------------------------------------------------------------- */
/* Local 8x8 block of one pair (T, T') summed over the outer points x_q:
 *   blk += omega * (gamma/2) * w_q * w_y * d d^T,
 *   d = (-phi_T(x_q) on T's nodes, +phi_T'(y) on T''s nodes),
 * at every inner quadrature point / accepted sample y (Eq. replaceBasis).   */
static void add_block(double blk[64], const double lx[4], const double v[4][3], const double y[3], double w)
{
    double lam[4], d[8];
    barycentric(v, y, lam);
    for (int a = 0; a < 4; ++a) { d[a] = -lx[a]; d[4 + a] = lam[a]; }
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) blk[8 * i + j] += w * d[i] * d[j];
}

/* accepted samples add omega (gamma/2) w_q (|S|/N) d d^T */
struct block_ctx {
    double *blk;
    const double *lx;
    const double (*v)[3];
    double coef;
    int acc;
    const double *kpoly;
    const double *x;
    double delta;
};

static void block_sample(void *p, int k, const double y[3], int cell, int accepted, double wgt)
{
    struct block_ctx *ctx = (struct block_ctx *)p;
    (void)k; (void)cell;
    if (!accepted) return;
    add_block(ctx->blk, ctx->lx, ctx->v, y, ctx->coef * (wgt * kshape(ctx->kpoly, ctx->x, y, ctx->delta)));
    ctx->acc++;
}

int or_pair_block(const double vT[12], const double vTp[12], double delta, double gamma,
                  int tp_in_collar, int strategy, int nmc, uint64_t seed,
                  uint32_t idT, uint32_t idTp, const double *kpoly, double blk[64])
{
    const double (*vt)[3] = (const double (*)[3])vT;
    const double (*v)[3] = (const double (*)[3])vTp;
    const int qmc = strategy == OR_FULLCAPS_QMC;
    if (qmc) strategy = OR_FULLCAPS;
    memset(blk, 0, sizeof(double) * 64);
    double xq[12];
    or_quad_points(vT, xq);
    double volT = or_tet_volume(vT);
    double omega = tp_in_collar ? 2.0 : 1.0;
    int acc = 0;
    for (int q = 0; q < 4; ++q) {
        const double *x = xq + 3 * q;
        double lx[4];
        barycentric(vt, x, lx);
        double coef = omega * (gamma / 2.0) * (volT / 4.0);
        classify_t c;
        classify(v, x, delta, &c);
        double cells[256][4][3];
        int nc = region_cells(v, x, delta, strategy, &c, cells, 256);
        for (int s = 0; s < nc; ++s) {
            double vol = tet_volume(cells[s][0], cells[s][1], cells[s][2], cells[s][3]);
            double flat[12], yq[12];
            memcpy(flat, cells[s], sizeof(flat));
            or_quad_points(flat, yq);
            for (int k = 0; k < 4; ++k)
                add_block(blk, lx, v, yq + 3 * k, coef * ((vol / 4.0) * kshape(kpoly, x, yq + 3 * k, delta)));
        }
        if (strategy == OR_FULLCAPS) {
            struct block_ctx bc = {blk, lx, v, coef, 0, kpoly, x, delta};
            cap_samples(v, vTp, x, delta, &c, nmc, seed, idT, idTp, (uint32_t)q, qmc, block_sample, &bc);
            acc += bc.acc;
        }
    }
    return acc;
}

/* The Monte Carlo samples of one (T', x) case as the assembly draws them:
 * y[3k..3k+2] the point, cell[k] its cap cell, accepted[k] = 1 when
 * |y - x|^2 <= delta^2 (arrays of nmc entries).  Returns the number of
 * samples drawn (0 when T' has no cap for x: all four vertices inside, or
 * T' not meeting the closed ball).                                          */
struct record_ctx {
    double *y;
    int32_t *cell;
    uint8_t *acc;
};

static void record_sample(void *p, int k, const double y[3], int cell, int accepted, double wgt)
{
    struct record_ctx *ctx = (struct record_ctx *)p;
    (void)wgt;
    ctx->y[3 * k] = y[0]; ctx->y[3 * k + 1] = y[1]; ctx->y[3 * k + 2] = y[2];
    ctx->cell[k] = cell;
    ctx->acc[k] = (uint8_t)accepted;
}

int or_cap_samples(const double vTp[12], const double x[3], double delta, int nmc, uint64_t seed,
                   uint32_t idT, uint32_t idTp, uint32_t q, double *y, int32_t *cell, uint8_t *accepted)
{
    const double (*v)[3] = (const double (*)[3])vTp;
    classify_t c;
    classify(v, x, delta, &c);
    struct record_ctx rc = {y, cell, accepted};
    return cap_samples(v, vTp, x, delta, &c, nmc, seed, idT, idTp, q, 0, record_sample, &rc);
}

int or_cap_samples_qmc(const double vTp[12], const double x[3], double delta, int nmc, uint64_t seed,
                       uint32_t idT, uint32_t idTp, uint32_t q, double *y, int32_t *cell, uint8_t *accepted)
{
    const double (*v)[3] = (const double (*)[3])vTp;
    classify_t c;
    classify(v, x, delta, &c);
    struct record_ctx rc = {y, cell, accepted};
    return cap_samples(v, vTp, x, delta, &c, nmc, seed, idT, idTp, q, 1, record_sample, &rc);
}

/* Blocks for a list of pairs (one 8x8 block per pair, rows/cols = the four
 * nodes of T then the four nodes of T').  Pairs are independent; each writes
 * only its own block, so the result does not depend on the thread count.  */
int64_t or_assemble_blocks(const double *verts, const int32_t *tets, const uint8_t *in_omega,
                           double delta, double gamma, int strategy, int nmc, uint64_t seed,
                           const double *kpoly, const int32_t *pT, const int32_t *pTp, int64_t npairs,
                           double *blocks, int nthreads)
{
    int64_t acc = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : acc)
#endif
    for (int64_t p = 0; p < npairs; ++p) {
        double vT[12], vTp[12];
        tet_coords(verts, tets, pT[p], vT);
        tet_coords(verts, tets, pTp[p], vTp);
        acc += or_pair_block(vT, vTp, delta, gamma, in_omega[pTp[p]] ? 0 : 1, strategy, nmc, seed,
                             (uint32_t)pT[p], (uint32_t)pTp[p], kpoly, blocks + 64 * p);
    }
    (void)nthreads;
    return acc;
}

/* Load vector F_i = sum_{T in Omega} sum_q w_q phi_i(x_q) f(x_q) (Eq. Fh with
 * the 4-point rule), f = fconst + the P1 interpolant of the nodal values
 * fnodal (NULL: constant f).                                                */
void or_load_vector(const double *verts, const int32_t *tets, int64_t nt, const uint8_t *in_omega,
                    int64_t nv, double fconst, const double *fnodal, double *F)
{
    memset(F, 0, sizeof(double) * (size_t)nv);
    for (int64_t t = 0; t < nt; ++t) {
        if (!in_omega[t]) continue;
        double v[12], xq[12];
        tet_coords(verts, tets, t, v);
        or_quad_points(v, xq);
        double w = or_tet_volume(v) / 4.0;
        for (int q = 0; q < 4; ++q) {
            double lam[4];
            barycentric((const double (*)[3])v, xq + 3 * q, lam);
            double f = fconst;
            if (fnodal)
                for (int a = 0; a < 4; ++a) f += lam[a] * fnodal[tets[4 * t + a]];
            for (int a = 0; a < 4; ++a) F[tets[4 * t + a]] += w * lam[a] * f;
        }
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
