// Per-(pair, outer point) inner moments of the approximate ball inside one
// element T' (Def. "simplex's dividing strategy", Def. "nocaps", the
// simplified 3D approxcaps of Sec. 3.3, fullcaps of Sec. 4.3.2 / Alg. 4).
//
// Moments are taken with respect to the barycentric coordinates lambda' of
// T':  m0 = |R|,  m1_a = int_R lambda'_a,  m2_ab = int_R lambda'_a lambda'_b.
// The cells of R are listed per case (number m of vertices inside the open
// ball) and integrated in closed form from the barycentric coordinates of
// their vertices (equal to the 4-point degree-2 rule, which is exact here).
//
// R = double: coordinates are global, x is the outer point; the translation
//             unit is compiled without fused multiply-add, so every decision
//             (inside test, edge/sphere point, diagonal, sampling volumes,
//             sample points and acceptance) follows the fixed operation order
//             of the method's arithmetic specification.
// R = float:  coordinates are relative to the outer point (x = 0).
#pragma once

#include <stdint.h>

namespace nlq {

template <class R> struct P3 { R x, y, z; };

template <class R> __device__ __forceinline__ P3<R> mk3(R x, R y, R z) { return P3<R>{x, y, z}; }
template <class R> __device__ __forceinline__ P3<R> sub(P3<R> a, P3<R> b) { return P3<R>{a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class R> __device__ __forceinline__ R dot(P3<R> a, P3<R> b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
template <class R> __device__ __forceinline__ R det3(P3<R> a, P3<R> b, P3<R> c)
{
    return (a.x * (b.y * c.z - b.z * c.y) + a.y * (b.z * c.x - b.x * c.z)) + a.z * (b.x * c.y - b.y * c.x);
}
template <class R> __device__ __forceinline__ R orient(P3<R> p0, P3<R> p1, P3<R> p2, P3<R> p3)
{
    return det3(sub(p1, p0), sub(p2, p0), sub(p3, p0));
}
template <class R> __device__ __forceinline__ R absr(R a) { return a < R(0) ? -a : a; }
template <class R> __device__ __forceinline__ R vol4(P3<R> p0, P3<R> p1, P3<R> p2, P3<R> p3)
{
    return absr(orient(p0, p1, p2, p3)) / R(6);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11)
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// uniforms in (0,1): FP64 (u + 0.5) 2^-32 (exact); FP32 ((u >> 8) + 0.5) 2^-24 (exact)
template <class R> __device__ __forceinline__ R unif(uint32_t u);
template <> __device__ __forceinline__ double unif<double>(uint32_t u) { return ((double)u + 0.5) * 0x1p-32; }
template <> __device__ __forceinline__ float unif<float>(uint32_t u) { return ((float)(u >> 8) + 0.5f) * 0x1p-24f; }
template <class R> __device__ __forceinline__ R unit_scale(uint32_t u);
template <> __device__ __forceinline__ double unit_scale<double>(uint32_t u) { return (double)u * 0x1p-32; }
template <> __device__ __forceinline__ float unit_scale<float>(uint32_t u) { return (float)(u >> 8) * 0x1p-24f; }

// ---------------------------------------------------------------------------
template <class R> struct Mom {
    R m0;
    R m1[4];
    R m2[10];     // (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3)
};

template <class R> __device__ __forceinline__ void mom_zero(Mom<R> &M)
{
    M.m0 = R(0);
#pragma unroll
    for (int a = 0; a < 4; ++a) M.m1[a] = R(0);
#pragma unroll
    for (int a = 0; a < 10; ++a) M.m2[a] = R(0);
}

// barycentric row of a point of the table: T' vertices 0..3 are unit rows;
// edge/sphere points are (1-t) e_i + t e_o
struct PDesc {
    int8_t i, o;   // for points >= 4
};

template <class R>
__device__ __forceinline__ void lam_row(int p, const PDesc *pd, const R *pt, R L[4])
{
#pragma unroll
    for (int a = 0; a < 4; ++a) L[a] = R(0);
    if (p < 4) {
#pragma unroll
        for (int a = 0; a < 4; ++a) L[a] = (a == p) ? R(1) : R(0);
    } else {
        int i = pd[p - 4].i, o = pd[p - 4].o;
        R t = pt[p - 4];
#pragma unroll
        for (int a = 0; a < 4; ++a) L[a] = (a == i) ? (R(1) - t) : ((a == o) ? t : R(0));
    }
}

// closed-form moments of one cell with vertex barycentric rows L0..L3
template <class R>
__device__ __forceinline__ void add_cell(Mom<R> &M, R vol, const R L0[4], const R L1[4], const R L2[4], const R L3[4])
{
    R S[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) S[a] = (L0[a] + L1[a]) + (L2[a] + L3[a]);
    R q4 = vol * R(0.25), q20 = vol * R(0.05);
    M.m0 += vol;
#pragma unroll
    for (int a = 0; a < 4; ++a) M.m1[a] += q4 * S[a];
    int k = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
            R s2 = ((L0[a] * L0[b] + L1[a] * L1[b]) + (L2[a] * L2[b] + L3[a] * L3[b])) + S[a] * S[b];
            M.m2[k++] += q20 * s2;
        }
}

// Squared distance from x to T' (zero inside): closest point on each face the
// point lies outside of.
template <class R> __device__ R d2_point_tri(P3<R> p, P3<R> a, P3<R> b, P3<R> c)
{
    P3<R> ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
    R d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= R(0) && d2 <= R(0)) return dot(ap, ap);
    P3<R> bp = sub(p, b);
    R d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= R(0) && d4 <= d3) return dot(bp, bp);
    R vc = d1 * d4 - d3 * d2;
    if (vc <= R(0) && d1 >= R(0) && d3 <= R(0)) {
        R v = d1 / (d1 - d3);
        P3<R> w = mk3<R>(ap.x - v * ab.x, ap.y - v * ab.y, ap.z - v * ab.z);
        return dot(w, w);
    }
    P3<R> cp = sub(p, c);
    R d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= R(0) && d5 <= d6) return dot(cp, cp);
    R vb = d5 * d2 - d1 * d6;
    if (vb <= R(0) && d2 >= R(0) && d6 <= R(0)) {
        R w = d2 / (d2 - d6);
        P3<R> r = mk3<R>(ap.x - w * ac.x, ap.y - w * ac.y, ap.z - w * ac.z);
        return dot(r, r);
    }
    R va = d3 * d6 - d5 * d4;
    if (va <= R(0) && (d4 - d3) >= R(0) && (d5 - d6) >= R(0)) {
        R w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        P3<R> r = mk3<R>(bp.x - w * (c.x - b.x), bp.y - w * (c.y - b.y), bp.z - w * (c.z - b.z));
        return dot(r, r);
    }
    R den = R(1) / ((va + vb) + vc);
    R v = vb * den, w = vc * den;
    P3<R> r = mk3<R>((ap.x - ab.x * v) - ac.x * w, (ap.y - ab.y * v) - ac.y * w, (ap.z - ab.z * v) - ac.z * w);
    return dot(r, r);
}

template <class R> __device__ R d2_point_tet(P3<R> p, const P3<R> v[4])
{
    R best = R(1e30);
    bool outside = false;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        int i0 = (f == 0) ? 1 : 0, i1 = (f <= 1) ? 2 : 1, i2 = (f <= 2) ? 3 : 2;
        P3<R> a = v[i0], b = v[i1], c = v[i2], o = v[f];
        R sp = det3(sub(b, a), sub(c, a), sub(p, a));
        R so = det3(sub(b, a), sub(c, a), sub(o, a));
        if ((sp < R(0) && so > R(0)) || (sp > R(0) && so < R(0))) {
            outside = true;
            R d = d2_point_tri(p, a, b, c);
            best = d < best ? d : best;
        }
    }
    return outside ? best : R(0);
}

// ---------------------------------------------------------------------------
// cell tables.  Points 0..3 are the vertices of T' by local index; points 4+
// are the edge/sphere points P(I[a], O[b]) at index 4 + a*(4-m) + b.
// "roles": r0..r3 = the inside vertices in increasing local index, then the
// outside vertices in increasing local index.  Entries < 4 below are roles.
#define NLQ_P(k) (4 + (k))
// cells of hull(I u P) (cone from the first inside vertex)
// m=1: (a, p0, p1, p2)
// m=2: c1=P0, d1=P1, c2=P2, d2=P3; diagonal c1-d2: (a,b,c2,d2) (a,c1,c2,d2) (a,c1,d2,d1)
//                                  diagonal c2-d1: (a,b,c2,d2) (a,c1,c2,d1) (a,c2,d2,d1)
// m=3: f1=P0, f2=P1, f3=P2: (a,f1,f2,f3) (a,b,c,f3) (a,b,f3,f2)
// cap cells S = T' \ hull(I u P) (the sampling order of the specification)
// m=1: (b,e1,e2,e3) (b,c,d,e3) (b,c,e3,e2)        [e_k = P(a, O[k])]
// m=2: (c,d,d1,d2) + diagonal c1-d2: (c,c1,c2,d2) (c,c1,d2,d1)
//                    diagonal c2-d1: (c,c1,c2,d1) (c,c2,d2,d1)
// m=3: (d, f1, f2, f3)

// ---------------------------------------------------------------------------
// Exact FP64 decisions for the FP32 path.  The FP32 kernel takes every
// decision (inside test, m=2 diagonal, cap cell choice, sample acceptance) in
// FP32 when it is clear by a wide margin, and otherwise recomputes it with the
// FP64 operations of the specification, written with explicit round-to-
// nearest intrinsics so that no multiply-add is fused.  The decisions of the
// FP32 path therefore equal those of the FP64 path.
struct Strict {
    double v[4][3];   // global coordinates of T'
    double x[3];      // outer point
    double d2;        // delta^2
};

__device__ __forceinline__ double sadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ssub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double smul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double sdot(const double a[3], const double b[3])
{
    return sadd(sadd(smul(a[0], b[0]), smul(a[1], b[1])), smul(a[2], b[2]));
}
__device__ __forceinline__ double sdet3(const double a[3], const double b[3], const double c[3])
{
    double t0 = smul(a[0], ssub(smul(b[1], c[2]), smul(b[2], c[1])));
    double t1 = smul(a[1], ssub(smul(b[2], c[0]), smul(b[0], c[2])));
    double t2 = smul(a[2], ssub(smul(b[0], c[1]), smul(b[1], c[0])));
    return sadd(sadd(t0, t1), t2);
}
__device__ __forceinline__ double sorient(const double p0[3], const double p1[3], const double p2[3],
                                          const double p3[3])
{
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) { e1[d] = ssub(p1[d], p0[d]); e2[d] = ssub(p2[d], p0[d]); e3[d] = ssub(p3[d], p0[d]); }
    return sdet3(e1, e2, e3);
}
__device__ __forceinline__ double svol4(const double p0[3], const double p1[3], const double p2[3],
                                        const double p3[3])
{
    return __ddiv_rn(fabs(sorient(p0, p1, p2, p3)), 6.0);
}
__device__ __forceinline__ double sr2(const double v[3], const double x[3])
{
    double w[3] = {ssub(v[0], x[0]), ssub(v[1], x[1]), ssub(v[2], x[2])};
    return sdot(w, w);
}
// edge/sphere point between an inside vertex vi and an outside vertex vo
__device__ __forceinline__ void sedge(const double vi[3], const double vo[3], const double x[3], double d2,
                                      double p[3])
{
    double w[3], e[3];
    for (int d = 0; d < 3; ++d) { w[d] = ssub(vi[d], x[d]); e[d] = ssub(vo[d], vi[d]); }
    double A = sdot(e, e), B = sdot(e, w), C = ssub(sdot(w, w), d2);
    double s = __dsqrt_rn(ssub(smul(B, B), smul(A, C)));
    double t = (B >= 0.0) ? __ddiv_rn(-C, sadd(B, s)) : __ddiv_rn(ssub(s, B), A);
    for (int d = 0; d < 3; ++d) p[d] = sadd(vi[d], smul(t, e[d]));
}

struct Stats {
    uint32_t cut, inside, mc, acc, fallback;
};

// Approximate-ball moments for one element T' and one outer point x.
//  v[4]  vertex coordinates (global for double, relative to x for float)
//  x     outer point (global for double, zero for float)
//  volTp |T'|
template <class R, int STRAT>
__device__ void point_moments(const P3<R> v[4], P3<R> x, R d2, R volTp, int nmc, uint2 key, uint32_t idT,
                              uint32_t idTp, uint32_t q, Mom<R> &M, Stats &st, const Strict *sx = nullptr)
{
    constexpr bool F32 = sizeof(R) == 4;
    const R MARGIN = R(1e-5);
    mom_zero(M);
    R r2[4];
    int inm = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        P3<R> w = sub(v[k], x);
        r2[k] = (w.x * w.x + w.y * w.y) + w.z * w.z;
        bool in = r2[k] < d2;
        if (F32 && sx && absr(r2[k] - d2) <= MARGIN * d2) in = sr2(sx->v[k], sx->x) < sx->d2;
        if (in) inm |= 1 << k;
    }
    const int m = __popc(inm);
    if (m == 4) {
        st.inside++;
        M.m0 = volTp;
        R q4 = volTp * R(0.25), q20 = volTp * R(0.05), q10 = volTp * R(0.1);
#pragma unroll
        for (int a = 0; a < 4; ++a) M.m1[a] = q4;
        M.m2[0] = q10; M.m2[1] = q20; M.m2[2] = q20; M.m2[3] = q20; M.m2[4] = q10;
        M.m2[5] = q20; M.m2[6] = q20; M.m2[7] = q10; M.m2[8] = q20; M.m2[9] = q10;
        return;
    }
    // roles
    int role[4];
    {
        int ni = 0, no = m;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (inm & (1 << k)) role[ni++] = k;
            else role[no++] = k;
        }
    }
    P3<R> pp[4];     // edge/sphere points
    R pt[4];         // their parameters
    PDesc pd[4];
    int np = 0;
    if (m > 0) {
        st.cut++;
        for (int a = 0; a < m; ++a)
            for (int b = m; b < 4; ++b) {
                int i = role[a], o = role[b];
                P3<R> w = sub(v[i], x);
                P3<R> e = sub(v[o], v[i]);
                R A = (e.x * e.x + e.y * e.y) + e.z * e.z;
                R B = (e.x * w.x + e.y * w.y) + e.z * w.z;
                R C = r2[i] - d2;
                R s = sqrt(B * B - A * C);
                R t = (B >= R(0)) ? (-C) / (B + s) : (s - B) / A;
                pp[np] = mk3<R>(v[i].x + t * e.x, v[i].y + t * e.y, v[i].z + t * e.z);
                pt[np] = t;
                pd[np].i = (int8_t)i;
                pd[np].o = (int8_t)o;
                np++;
            }
    }
    // point lookup: p < 4 -> vertex by local index, else edge point
    auto P = [&](int p) -> P3<R> { return p < 4 ? v[p] : pp[p - 4]; };

    bool diag_c2d1 = false;
    if (m == 2) {
        P3<R> c1 = pp[0], d1 = pp[1], c2 = pp[2], dd2 = pp[3];
        R o1 = orient(c1, c2, dd2, d1), o2 = orient(c1, c2, dd2, v[role[0]]);
        if (F32 && sx) {
            P3<R> e = sub(v[role[2]], v[role[0]]);
            R L = (absr(e.x) + absr(e.y)) + absr(e.z);
            R tol = R(1e-4) * L * L * L;
            if (absr(o1) <= tol || absr(o2) <= tol) {
                double P64[4][3];
                sedge(sx->v[role[0]], sx->v[role[2]], sx->x, sx->d2, P64[0]);
                sedge(sx->v[role[0]], sx->v[role[3]], sx->x, sx->d2, P64[1]);
                sedge(sx->v[role[1]], sx->v[role[2]], sx->x, sx->d2, P64[2]);
                sedge(sx->v[role[1]], sx->v[role[3]], sx->x, sx->d2, P64[3]);
                double q1 = sorient(P64[0], P64[2], P64[3], P64[1]);
                double q2 = sorient(P64[0], P64[2], P64[3], sx->v[role[0]]);
                o1 = q1 > 0.0 ? R(1) : (q1 < 0.0 ? R(-1) : R(0));
                o2 = q2 > 0.0 ? R(1) : (q2 < 0.0 ? R(-1) : R(0));
            }
        }
        diag_c2d1 = (o1 > R(0) && o2 < R(0)) || (o1 < R(0) && o2 > R(0));
    }

    // deterministic cells: hull(I u P)
    if (m > 0) {
        int cells[3][4];
        int nc = 0;
        const int a = role[0];
        if (m == 1) {
            cells[0][0] = a; cells[0][1] = NLQ_P(0); cells[0][2] = NLQ_P(1); cells[0][3] = NLQ_P(2);
            nc = 1;
        } else if (m == 2) {
            const int b = role[1];
            cells[0][0] = a; cells[0][1] = b; cells[0][2] = NLQ_P(2); cells[0][3] = NLQ_P(3);
            if (!diag_c2d1) {
                cells[1][0] = a; cells[1][1] = NLQ_P(0); cells[1][2] = NLQ_P(2); cells[1][3] = NLQ_P(3);
                cells[2][0] = a; cells[2][1] = NLQ_P(0); cells[2][2] = NLQ_P(3); cells[2][3] = NLQ_P(1);
            } else {
                cells[1][0] = a; cells[1][1] = NLQ_P(0); cells[1][2] = NLQ_P(2); cells[1][3] = NLQ_P(1);
                cells[2][0] = a; cells[2][1] = NLQ_P(2); cells[2][2] = NLQ_P(3); cells[2][3] = NLQ_P(1);
            }
            nc = 3;
        } else {
            const int b = role[1], c = role[2];
            cells[0][0] = a; cells[0][1] = NLQ_P(0); cells[0][2] = NLQ_P(1); cells[0][3] = NLQ_P(2);
            cells[1][0] = a; cells[1][1] = b; cells[1][2] = c; cells[1][3] = NLQ_P(2);
            cells[2][0] = a; cells[2][1] = b; cells[2][2] = NLQ_P(2); cells[2][3] = NLQ_P(1);
            nc = 3;
        }
        for (int j = 0; j < nc; ++j) {
            R L0[4], L1[4], L2[4], L3[4];
            lam_row<R>(cells[j][0], pd, pt, L0);
            lam_row<R>(cells[j][1], pd, pt, L1);
            lam_row<R>(cells[j][2], pd, pt, L2);
            lam_row<R>(cells[j][3], pd, pt, L3);
            R vol = vol4(P(cells[j][0]), P(cells[j][1]), P(cells[j][2]), P(cells[j][3]));
            add_cell(M, vol, L0, L1, L2, L3);
        }
    }

    if (STRAT == 2 && nmc > 0) {
        bool run = (m > 0);
        if (!run) {
            R dd = d2_point_tet(x, v);
            run = dd <= d2;
            if (F32 && sx && absr(dd - d2) <= R(1e-4) * d2) {
                P3<double> vd[4];
                for (int k = 0; k < 4; ++k) vd[k] = mk3<double>(sx->v[k][0], sx->v[k][1], sx->v[k][2]);
                run = d2_point_tet(mk3<double>(sx->x[0], sx->x[1], sx->x[2]), vd) <= sx->d2;
            }
        }
        if (run) {
            int S[3][4];
            int ns;
            if (m == 0) {
                S[0][0] = 0; S[0][1] = 1; S[0][2] = 2; S[0][3] = 3;
                ns = 1;
            } else if (m == 1) {
                const int b = role[1], c = role[2], d = role[3];
                S[0][0] = b; S[0][1] = NLQ_P(0); S[0][2] = NLQ_P(1); S[0][3] = NLQ_P(2);
                S[1][0] = b; S[1][1] = c; S[1][2] = d; S[1][3] = NLQ_P(2);
                S[2][0] = b; S[2][1] = c; S[2][2] = NLQ_P(2); S[2][3] = NLQ_P(1);
                ns = 3;
            } else if (m == 2) {
                const int c = role[2], d = role[3];
                S[0][0] = c; S[0][1] = d; S[0][2] = NLQ_P(1); S[0][3] = NLQ_P(3);
                if (!diag_c2d1) {
                    S[1][0] = c; S[1][1] = NLQ_P(0); S[1][2] = NLQ_P(2); S[1][3] = NLQ_P(3);
                    S[2][0] = c; S[2][1] = NLQ_P(0); S[2][2] = NLQ_P(3); S[2][3] = NLQ_P(1);
                } else {
                    S[1][0] = c; S[1][1] = NLQ_P(0); S[1][2] = NLQ_P(2); S[1][3] = NLQ_P(1);
                    S[2][0] = c; S[2][1] = NLQ_P(2); S[2][2] = NLQ_P(3); S[2][3] = NLQ_P(1);
                }
                ns = 3;
            } else {
                const int d = role[3];
                S[0][0] = d; S[0][1] = NLQ_P(0); S[0][2] = NLQ_P(1); S[0][3] = NLQ_P(2);
                ns = 1;
            }
            P3<R> sp[3][4];
            R sl[3][4][4];
            R vol[3];
            R tot = R(0);
            for (int j = 0; j < ns; ++j) {
                for (int k = 0; k < 4; ++k) {
                    sp[j][k] = P(S[j][k]);
                    lam_row<R>(S[j][k], pd, pt, sl[j][k]);
                }
                vol[j] = vol4(sp[j][0], sp[j][1], sp[j][2], sp[j][3]);
            }
            for (int j = 0; j < ns; ++j) tot += vol[j];
            R a0 = R(0), a1[4] = {R(0), R(0), R(0), R(0)}, a2[10];
#pragma unroll
            for (int k = 0; k < 10; ++k) a2[k] = R(0);
            uint32_t acc = 0;
            // FP64 cap cells for samples whose FP32 decision is within the margin
            bool have64 = false;
            double s64[3][4][3], vol64[3], tot64 = 0.0;
            auto build64 = [&]() {
                double P64[4][3];
                for (int n = 0; n < np; ++n)
                    sedge(sx->v[pd[n].i], sx->v[pd[n].o], sx->x, sx->d2, P64[n]);
                for (int jj = 0; jj < ns; ++jj) {
                    for (int kk = 0; kk < 4; ++kk) {
                        int pidx = S[jj][kk];
                        for (int d = 0; d < 3; ++d) s64[jj][kk][d] = pidx < 4 ? sx->v[pidx][d] : P64[pidx - 4][d];
                    }
                    vol64[jj] = svol4(s64[jj][0], s64[jj][1], s64[jj][2], s64[jj][3]);
                }
                tot64 = 0.0;
                for (int jj = 0; jj < ns; ++jj) tot64 = sadd(tot64, vol64[jj]);
                have64 = true;
            };
            for (int k = 0; k < nmc; ++k) {
                uint4 u = philox4x32_10(make_uint4(idT, idTp, q, (uint32_t)k), key);
                R r = unit_scale<R>(u.x) * tot;
                int j = ns - 1;
                R cum = R(0);
                bool unsure = false;
                for (int jj = 0; jj < ns; ++jj) {
                    cum += vol[jj];
                    if (F32 && jj < ns - 1 && absr(r - cum) <= MARGIN * tot) unsure = true;
                    if (r < cum) { j = jj; break; }
                }
                R U0 = unif<R>(u.y), U1 = unif<R>(u.z), U2 = unif<R>(u.w), tmp;
                if (U0 > U1) { tmp = U0; U0 = U1; U1 = tmp; }
                if (U1 > U2) { tmp = U1; U1 = U2; U2 = tmp; }
                if (U0 > U1) { tmp = U0; U0 = U1; U1 = tmp; }
                R be0 = U0, be1 = U1 - U0, be2 = U2 - U1, be3 = R(1) - U2;
                P3<R> s0 = sp[j][0], s1 = sp[j][1], s2 = sp[j][2], s3 = sp[j][3];
                P3<R> y = mk3<R>(((be0 * s0.x + be1 * s1.x) + be2 * s2.x) + be3 * s3.x,
                                 ((be0 * s0.y + be1 * s1.y) + be2 * s2.y) + be3 * s3.y,
                                 ((be0 * s0.z + be1 * s1.z) + be2 * s2.z) + be3 * s3.z);
                P3<R> w = sub(y, x);
                R rr = (w.x * w.x + w.y * w.y) + w.z * w.z;
                bool inb = rr <= d2;
                if (F32 && sx && (unsure || absr(rr - d2) <= MARGIN * d2)) {
                    // the specification's FP64 sample: cell by cumulative volume, exact
                    // spacings of the 32-bit uniforms, point and ball test
                    if (!have64) build64();
                    double rd = smul((double)u.x * 0x1p-32, tot64);
                    int j64 = ns - 1;
                    double c64 = 0.0;
                    for (int jj = 0; jj < ns; ++jj) {
                        c64 = sadd(c64, vol64[jj]);
                        if (rd < c64) { j64 = jj; break; }
                    }
                    double V0 = ((double)u.y + 0.5) * 0x1p-32, V1 = ((double)u.z + 0.5) * 0x1p-32,
                           V2 = ((double)u.w + 0.5) * 0x1p-32, tv;
                    if (V0 > V1) { tv = V0; V0 = V1; V1 = tv; }
                    if (V1 > V2) { tv = V1; V1 = V2; V2 = tv; }
                    if (V0 > V1) { tv = V0; V0 = V1; V1 = tv; }
                    double b0 = V0, b1 = ssub(V1, V0), b2 = ssub(V2, V1), b3 = ssub(1.0, V2);
                    double wy[3];
                    for (int d = 0; d < 3; ++d) {
                        double yd = sadd(sadd(sadd(smul(b0, s64[j64][0][d]), smul(b1, s64[j64][1][d])),
                                              smul(b2, s64[j64][2][d])),
                                         smul(b3, s64[j64][3][d]));
                        wy[d] = ssub(yd, sx->x[d]);
                    }
                    inb = sdot(wy, wy) <= sx->d2;
                    j = j64;
                }
                if (inb) {
                    R lam[4];
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa)
                        lam[aa] = ((be0 * sl[j][0][aa] + be1 * sl[j][1][aa]) + be2 * sl[j][2][aa]) + be3 * sl[j][3][aa];
                    acc++;
                    a0 += R(1);
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa) a1[aa] += lam[aa];
                    int kk = 0;
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa)
#pragma unroll
                        for (int bb = aa; bb < 4; ++bb) a2[kk++] += lam[aa] * lam[bb];
                }
            }
            st.mc += (uint32_t)nmc;
            st.acc += acc;
            R wgt = tot / R(nmc);
            M.m0 += wgt * a0;
#pragma unroll
            for (int aa = 0; aa < 4; ++aa) M.m1[aa] += wgt * a1[aa];
#pragma unroll
            for (int kk = 0; kk < 10; ++kk) M.m2[kk] += wgt * a2[kk];
        }
    }
}

}  // namespace nlq
