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
#include <type_traits>

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

// Uniforms.  FP64: U = (u + 0.5) 2^-32 in (0,1) and u 2^-32 in [0,1), both
// exact.  FP32: the top 23 bits, U = (k + 0.5) 2^-23 and k 2^-23 with
// k = u >> 9, built from the bit pattern of 1 + k 2^-23 (exact, and no
// integer-to-float conversion instruction).  The FP32 values differ from the
// FP64 ones by less than 2^-23; decisions within the FP32 margins are
// retaken with the FP64 values.
template <class R> __device__ __forceinline__ R unif(uint32_t u);
template <> __device__ __forceinline__ double unif<double>(uint32_t u) { return ((double)u + 0.5) * 0x1p-32; }
template <> __device__ __forceinline__ float unif<float>(uint32_t u)
{
    return __uint_as_float(0x3f800000u | (u >> 9)) - (1.0f - 0x1p-24f);
}
template <class R> __device__ __forceinline__ R unit_scale(uint32_t u);
template <> __device__ __forceinline__ double unit_scale<double>(uint32_t u) { return (double)u * 0x1p-32; }
template <> __device__ __forceinline__ float unit_scale<float>(uint32_t u)
{
    return __uint_as_float(0x3f800000u | (u >> 9)) - 1.0f;
}

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

// Kernel shape phi(|x - y|): the kernel is gamma phi (Sec. 2; the constant
// kernel is phi = 1).  KerConst: phi = 1, integrated in closed form.
// KerShape: phi = c0 + c1 s + c2 s^2 + c3 s^3 in s = min(|x - y|^2 / delta^2,
// 1) (the element-level strategies place points past the sphere, where phi
// keeps its value on it); cells then take the 4-point rule with phi at the
// rule points (Sec. 4.3.1), and accepted cap samples are weighted by phi.
struct KerConst {
    static constexpr bool constant = true;
};
template <class R> struct KerShape {
    static constexpr bool constant = false;
    R c0, c1, c2, c3, d2;
    // phi at squared distance rr
    __device__ __forceinline__ R operator()(R rr) const
    {
        R s = rr / d2;
        s = s < R(1) ? s : R(1);
        return c0 + s * (c1 + s * (c2 + s * c3));
    }
};

// The weight of an accepted cap sample at squared distance rr
template <class R, class KER> __device__ __forceinline__ R kweight(const KER &ker, R rr)
{
    if constexpr (KER::constant) {
        (void)ker; (void)rr;
        return R(1);
    } else {
        return ker(rr);
    }
}

// The 4-point rule's weights a (own vertex) and b (the others)
template <class R> __device__ __forceinline__ R rule_a() { return R(0x1.2bbae2a27f931p-1); }
template <class R> __device__ __forceinline__ R rule_b() { return R(0x1.1b06d1d200913p-3); }

// Moments of one cell with vertex barycentric rows L0..L3 and vertices
// p0..p3: closed form for the constant kernel, else the 4-point rule with the
// kernel shape at the rule points y_k = b (p0 + p1 + p2 + p3) + (a - b) p_k,
// where lambda' = b (L0 + L1 + L2 + L3) + (a - b) L_k.
template <class R, class KER>
__device__ __forceinline__ void add_cell_k(Mom<R> &M, R vol, const R L0[4], const R L1[4], const R L2[4],
                                           const R L3[4], P3<R> p0, P3<R> p1, P3<R> p2, P3<R> p3, P3<R> x,
                                           const KER &ker)
{
    if constexpr (KER::constant) {
        (void)p0; (void)p1; (void)p2; (void)p3; (void)x; (void)ker;
        add_cell(M, vol, L0, L1, L2, L3);
    } else {
        const R qa = rule_a<R>(), qb = rule_b<R>(), qd = qa - qb;
        const P3<R> ps = mk3<R>((p0.x + p1.x) + (p2.x + p3.x), (p0.y + p1.y) + (p2.y + p3.y),
                                (p0.z + p1.z) + (p2.z + p3.z));
        R S[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) S[a] = (L0[a] + L1[a]) + (L2[a] + L3[a]);
        const P3<R> pk[4] = {p0, p1, p2, p3};
        const R *Lk[4] = {L0, L1, L2, L3};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const P3<R> w = mk3<R>(qb * ps.x + qd * pk[k].x - x.x, qb * ps.y + qd * pk[k].y - x.y,
                                   qb * ps.z + qd * pk[k].z - x.z);
            const R f = (vol * R(0.25)) * ker((w.x * w.x + w.y * w.y) + w.z * w.z);
            R lam[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) lam[a] = qb * S[a] + qd * Lk[k][a];
            M.m0 += f;
#pragma unroll
            for (int a = 0; a < 4; ++a) M.m1[a] += f * lam[a];
            int t = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = a; b < 4; ++b) M.m2[t++] += (f * lam[a]) * lam[b];
        }
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
    const double4 *verts;   // global vertex table (FP64)
    int4 e;                 // vertex ids of T'
    const double *x;        // outer point, 3 doubles
    double d2;              // delta^2
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

__device__ __forceinline__ void strict_load(const Strict *sx, double v[4][3], double x[3])
{
    const int ids[4] = {sx->e.x, sx->e.y, sx->e.z, sx->e.w};
    for (int k = 0; k < 4; ++k) {
        double4 g = sx->verts[ids[k]];
        v[k][0] = g.x; v[k][1] = g.y; v[k][2] = g.z;
    }
    x[0] = sx->x[0]; x[1] = sx->x[1]; x[2] = sx->x[2];
}

// FP64 inside test of vertex k (specification order).
static __device__ __noinline__ bool strict_inside(const Strict *sx, int k)
{
    double v[4][3], x[3];
    strict_load(sx, v, x);
    return sr2(v[k], x) < sx->d2;
}

// FP64 m=2 diagonal: true for the c2-d1 diagonal.
static __device__ __noinline__ bool strict_diag(const Strict *sx, int r0, int r1, int r2, int r3)
{
    double v[4][3], x[3];
    strict_load(sx, v, x);
    double P64[4][3];
    sedge(v[r0], v[r2], x, sx->d2, P64[0]);
    sedge(v[r0], v[r3], x, sx->d2, P64[1]);
    sedge(v[r1], v[r2], x, sx->d2, P64[2]);
    sedge(v[r1], v[r3], x, sx->d2, P64[3]);
    double q1 = sorient(P64[0], P64[2], P64[3], P64[1]);
    double q2 = sorient(P64[0], P64[2], P64[3], v[r0]);
    return (q1 > 0.0 && q2 < 0.0) || (q1 < 0.0 && q2 > 0.0);
}

// FP64 data of one event's cap built on the first exact decision: the edge
// points and the cell volumes (local memory; used only on that rare path).
struct StrictCap {
    int ready;
    double P[4][3];
    double vol[3];
    double tot;
};

// Cube root of a > 0 by Newton's method, x <- x - (x^3 - a) / (3 x^2), six
// steps from 2^q (1 + (m 2^r - 1) / 3) where a = m 2^(3q + r), m in
// [0.5, 1), r in {0, 1, 2} (the start is within 0.2 of the root's mantissa;
// six quadratic steps reach double precision).  Every operation rounded on
// its own, so that the value does not depend on the translation unit.
__device__ __forceinline__ double cbrt_newton(double a)
{
    int e;
    const double m = frexp(a, &e);
    int q = e / 3, r = e - 3 * q;
    if (r < 0) { r += 3; q -= 1; }
    double x = ldexp(__dadd_rn(1.0, __ddiv_rn(__dsub_rn(ldexp(m, r), 1.0), 3.0)), q);
    for (int i = 0; i < 6; ++i) {
        const double xx = __dmul_rn(x, x);
        x = __dsub_rn(x, __ddiv_rn(__dsub_rn(__dmul_rn(xx, x), a), __dmul_rn(3.0, xx)));
    }
    return x;
}

// The specification's FP64 sample for the words u.  The cap cells are
// described by their packed point indices (3 bits per point, 4 points per
// cell, ns cells) and the edge points (2+2 bits: inside, outside vertex).
// The point: sorted uniforms (Monte Carlo), or with qmc the nested map
// s = U1^(1/3), t = U2^(1/2), w = U3, beta = (1 - s, s (1 - t),
// s t (1 - w), s t w).
static __device__ __noinline__ int strict_sample(const Strict *sx, StrictCap *cap, unsigned long long spack, int ns,
                                                 uint32_t pdpack, int np, uint4 u, int *jout, int qmc = 0)
{
    double v[4][3], x[3];
    strict_load(sx, v, x);
    if (!cap->ready) {
        for (int n = 0; n < np; ++n) {
            int i = (pdpack >> (4 * n)) & 3, o = (pdpack >> (4 * n + 2)) & 3;
            sedge(v[i], v[o], x, sx->d2, cap->P[n]);
        }
        double tot = 0.0;
        for (int jj = 0; jj < ns; ++jj) {
            const double *c[4];
            for (int kk = 0; kk < 4; ++kk) {
                int pidx = (int)((spack >> (3 * (4 * jj + kk))) & 7);
                c[kk] = pidx < 4 ? v[pidx] : cap->P[pidx - 4];
            }
            cap->vol[jj] = svol4(c[0], c[1], c[2], c[3]);
            tot = sadd(tot, cap->vol[jj]);
        }
        cap->tot = tot;
        cap->ready = 1;
    }
    double rd = smul((double)u.x * 0x1p-32, cap->tot);
    int j64 = ns - 1;
    double c64 = 0.0;
    for (int jj = 0; jj < ns; ++jj) {
        c64 = sadd(c64, cap->vol[jj]);
        if (rd < c64) { j64 = jj; break; }
    }
    double V0 = ((double)u.y + 0.5) * 0x1p-32, V1 = ((double)u.z + 0.5) * 0x1p-32, V2 = ((double)u.w + 0.5) * 0x1p-32,
           tv;
    double b0, b1, b2, b3;
    if (qmc) {
        const double sc = cbrt_newton(V0), tc = __dsqrt_rn(V1), st = smul(sc, tc);
        b0 = ssub(1.0, sc); b1 = smul(sc, ssub(1.0, tc)); b2 = smul(st, ssub(1.0, V2)); b3 = smul(st, V2);
    } else {
        if (V0 > V1) { tv = V0; V0 = V1; V1 = tv; }
        if (V1 > V2) { tv = V1; V1 = V2; V2 = tv; }
        if (V0 > V1) { tv = V0; V0 = V1; V1 = tv; }
        b0 = V0; b1 = ssub(V1, V0); b2 = ssub(V2, V1); b3 = ssub(1.0, V2);
    }
    const double *c[4];
    for (int kk = 0; kk < 4; ++kk) {
        int pidx = (int)((spack >> (3 * (4 * j64 + kk))) & 7);
        c[kk] = pidx < 4 ? v[pidx] : cap->P[pidx - 4];
    }
    double wy[3];
    for (int d = 0; d < 3; ++d) {
        double yd = sadd(sadd(sadd(smul(b0, c[0][d]), smul(b1, c[1][d])), smul(b2, c[2][d])), smul(b3, c[3][d]));
        wy[d] = ssub(yd, x[d]);
    }
    *jout = j64;
    return sdot(wy, wy) <= sx->d2 ? 1 : 0;
}

// FP64 barycenter test of the specification: the centroid
// 0.25 ((v0 + v1) + (v2 + v3)) in the closed ball.
static __device__ __noinline__ bool strict_bary(const Strict *sx)
{
    double v[4][3], x[3], w[3];
    strict_load(sx, v, x);
    for (int d = 0; d < 3; ++d) w[d] = ssub(smul(0.25, sadd(sadd(v[0][d], v[1][d]), sadd(v[2][d], v[3][d]))), x[d]);
    return sdot(w, w) <= sx->d2;
}

static __device__ __noinline__ bool strict_meets(const Strict *sx)
{
    double v[4][3], x[3];
    strict_load(sx, v, x);
    P3<double> vd[4];
    for (int k = 0; k < 4; ++k) vd[k] = mk3<double>(v[k][0], v[k][1], v[k][2]);
    return d2_point_tet(mk3<double>(x[0], x[1], x[2]), vd) <= sx->d2;
}

struct Stats {
    uint32_t cut, inside, mc, acc, fallback;
};

// ---------------------------------------------------------------------------
// Classification of the four vertices of T' against the open ball around x
// (Def. simplex's dividing strategy): bit k of the result is set when
// |v_k - x|^2 < delta^2.  The FP32 path decides within a 1e-5 relative margin
// of the sphere with the FP64 specification (sx).
template <class R>
__device__ __forceinline__ int classify(const P3<R> v[4], P3<R> x, R d2, const Strict *sx)
{
    constexpr bool F32 = sizeof(R) == 4;
    int inm = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        P3<R> w = sub(v[k], x);
        R r2 = (w.x * w.x + w.y * w.y) + w.z * w.z;
        bool in = r2 < d2;
        if (F32 && sx && absr(r2 - d2) <= R(1e-5) * d2) in = strict_inside(sx, k);
        if (in) inm |= 1 << k;
    }
    return inm;
}

// Whether T' meets the closed ball when no vertex is inside (the fullcaps
// cap of Alg. 4 exists only then).
template <class R>
__device__ __forceinline__ bool meets_ball(const P3<R> v[4], P3<R> x, R d2, const Strict *sx)
{
    constexpr bool F32 = sizeof(R) == 4;
    if constexpr (F32) {
        // branch-free decisions far from the sphere (relative margin 1e-4 on
        // squared distances, far above the FP32 rounding): a bounding sphere
        // of T' (centroid, farthest vertex) that misses the ball, or an edge
        // of T' with a point inside the ball (any point of the segment gives
        // an upper bound of the distance, so the clamped parameter need not
        // be exact)
        const P3<R> c = mk3<R>(R(0.25) * ((v[0].x + v[1].x) + (v[2].x + v[3].x)),
                               R(0.25) * ((v[0].y + v[1].y) + (v[2].y + v[3].y)),
                               R(0.25) * ((v[0].z + v[1].z) + (v[2].z + v[3].z)));
        R rad2 = R(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const P3<R> w = sub(v[k], c);
            const R r2 = dot(w, w);
            rad2 = r2 > rad2 ? r2 : rad2;
        }
        const P3<R> wc = sub(c, x);
        const R reach = sqrt(d2) + sqrt(rad2);
        if (dot(wc, wc) > reach * reach * R(1.0001)) return false;
        R emin = R(3.0e38);
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const int i = e < 3 ? 0 : (e < 5 ? 1 : 2);
            const int j = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
            const P3<R> ab = sub(v[j], v[i]), ap = sub(x, v[i]);
            R t = __fdividef(dot(ap, ab), dot(ab, ab));
            t = t < R(0) ? R(0) : (t > R(1) ? R(1) : t);
            const P3<R> r = mk3<R>(ap.x - t * ab.x, ap.y - t * ab.y, ap.z - t * ab.z);
            const R e2 = dot(r, r);
            emin = e2 < emin ? e2 : emin;
        }
        if (emin < d2 * R(0.9999)) return true;
    }
    R dd = d2_point_tet(x, v);
    bool run = dd <= d2;
    if (F32 && sx && absr(dd - d2) <= R(1e-4) * d2) run = strict_meets(sx);
    return run;
}

// The element-level approximate balls of Sec. 4.3 take T' whole or not at
// all (STRAT 3 barycenter: the centroid in the closed ball; 4 overlap: T'
// meets the closed ball; 5 inside: every vertex in the open ball).  inm is
// the vertex classification; the FP32 path retakes close decisions in FP64.
template <class R, int STRAT>
__device__ __forceinline__ bool element_full(const P3<R> v[4], P3<R> x, R d2, int inm, const Strict *sx)
{
    constexpr bool F32 = sizeof(R) == 4;
    if (STRAT == 5) return inm == 15;
    if (STRAT == 4) return inm != 0 || meets_ball(v, x, d2, sx);
    P3<R> w;
    w.x = R(0.25) * ((v[0].x + v[1].x) + (v[2].x + v[3].x)) - x.x;
    w.y = R(0.25) * ((v[0].y + v[1].y) + (v[2].y + v[3].y)) - x.y;
    w.z = R(0.25) * ((v[0].z + v[1].z) + (v[2].z + v[3].z)) - x.z;
    const R r2 = (w.x * w.x + w.y * w.y) + w.z * w.z;
    if (F32 && sx && absr(r2 - d2) <= R(1e-5) * d2) return strict_bary(sx);
    return r2 <= d2;
}

template <class R> __device__ __forceinline__ void closed_form_inside(Mom<R> &M, R volTp)
{
    M.m0 = volTp;
    R q4 = volTp * R(0.25), q20 = volTp * R(0.05), q10 = volTp * R(0.1);
#pragma unroll
    for (int a = 0; a < 4; ++a) M.m1[a] = q4;
    M.m2[0] = q10; M.m2[1] = q20; M.m2[2] = q20; M.m2[3] = q20; M.m2[4] = q10;
    M.m2[5] = q20; M.m2[6] = q20; M.m2[7] = q10; M.m2[8] = q20; M.m2[9] = q10;
}

// Moments of the whole T' (volume volTp) under a kernel shape: the 4-point
// rule on T', whose rule points have lambda' = (a on vertex k, b elsewhere).
template <class R>
__device__ __forceinline__ void whole_moments(const P3<R> v[4], P3<R> x, R volTp, const KerShape<R> &ker, Mom<R> &M)
{
    mom_zero(M);
    R L[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int a = 0; a < 4; ++a) L[k][a] = (a == k) ? R(1) : R(0);
    add_cell_k(M, volTp, L[0], L[1], L[2], L[3], v[0], v[1], v[2], v[3], x, ker);
}

// Philox with the per-round keys precomputed (rk[2r], rk[2r+1] = key + r*Weyl).
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

// ---------------------------------------------------------------------------
// Quasi-Monte Carlo cap points (NL_FULLCAPS_QMC; better sampling over the
// caps is left open by Sec. 4.3.2): Sobol' points (Sobol' 1967) in four
// dimensions, each word XORed with a per-event random word (a digital shift:
// every point stays uniform on the 2^32 grid, the net structure stays).
// Direction numbers: v_b = m_{b+1} 2^(31-b) with, in dimension 0, m_k = 1
// (van der Corput), and in dimensions 1..3 the primitive polynomials
// x + 1, x^2 + x + 1, x^3 + x + 1 with initial m = (1), (1, 3), (1, 3, 1)
// (Joe & Kuo's table, 2008) continued by Sobol's recurrence
//   m_k = m_{k-s} ^ (m_{k-s} << s) ^ sum_{i<s, a_i = 1} (m_{k-i} << i).
// Sample k takes the point of Gray-code index k ^ (k >> 1), so that point
// k is point k-1 XOR the direction of the lowest set bit of k.
struct SobolDirs {
    uint32_t v[4][32];
};

constexpr SobolDirs make_sobol_dirs()
{
    SobolDirs d{};
    const int deg[4] = {0, 1, 2, 3};
    const unsigned inner[4] = {0u, 0u, 1u, 1u};   // a_1 .. a_{s-1}, a_1 the high bit
    const uint32_t init[4][3] = {{0u, 0u, 0u}, {1u, 0u, 0u}, {1u, 3u, 0u}, {1u, 3u, 1u}};
    for (int b = 0; b < 32; ++b) d.v[0][b] = 1u << (31 - b);
    for (int dim = 1; dim < 4; ++dim) {
        const int sdeg = deg[dim];
        uint32_t m[33] = {};
        for (int k = 1; k <= sdeg; ++k) m[k] = init[dim][k - 1];
        for (int k = sdeg + 1; k <= 32; ++k) {
            uint32_t x = m[k - sdeg] ^ (m[k - sdeg] << sdeg);
            for (int i = 1; i < sdeg; ++i)
                if ((inner[dim] >> (sdeg - 1 - i)) & 1u) x ^= m[k - i] << i;
            m[k] = x;
        }
        for (int b = 0; b < 32; ++b) d.v[dim][b] = m[b + 1] << (31 - b);
    }
    return d;
}

static __constant__ SobolDirs kSobol = make_sobol_dirs();

// The words of one event's samples in order k = 0, 1, ...: Philox draws of
// counter (T, T', q, k), or (QMC) Sobol' points XOR the Philox draw of
// counter (T, T', q, 0xFFFFFFFF).
template <bool QMC>
struct CapDraws {
    uint32_t idT, idTp, q;
    const uint32_t *rk;
    uint4 shift, pt;
    __device__ __forceinline__ CapDraws(uint32_t a, uint32_t b, uint32_t c, const uint32_t *keys)
        : idT(a), idTp(b), q(c), rk(keys), shift(make_uint4(0u, 0u, 0u, 0u)), pt(make_uint4(0u, 0u, 0u, 0u))
    {
        if constexpr (QMC) shift = philox_rk(make_uint4(idT, idTp, q, 0xFFFFFFFFu), rk);
    }
    // the k-th words; with QMC, calls must come in order k = 0, 1, ...
    __device__ __forceinline__ uint4 next(int k)
    {
        if constexpr (QMC) {
            if (k > 0) {
                const int b = __ffs(k) - 1;
                pt.x ^= kSobol.v[0][b]; pt.y ^= kSobol.v[1][b]; pt.z ^= kSobol.v[2][b]; pt.w ^= kSobol.v[3][b];
            }
            return make_uint4(pt.x ^ shift.x, pt.y ^ shift.y, pt.z ^ shift.z, pt.w ^ shift.w);
        } else {
            return philox_rk(make_uint4(idT, idTp, q, (uint32_t)k), rk);
        }
    }
};

// Barycentric coordinates of a cap sample in its cell from the words u
// (u.y, u.z, u.w): Monte Carlo takes the spacings of the three sorted
// uniforms; quasi-Monte Carlo the nested map s = U1^(1/3), t = U2^(1/2),
// w = U3, beta = (1 - s, s (1 - t), s t (1 - w), s t w), continuous in the
// uniforms as low-discrepancy points need (FP32: CUDA's cbrtf; FP64: the
// Newton cube root of the specification).
template <class R, bool QMC>
__device__ __forceinline__ void cap_bary(uint4 u, R &b0, R &b1, R &b2, R &b3)
{
    const R U2 = unif<R>(u.w);
    if constexpr (QMC) {
        R sc, tc;
        if constexpr (sizeof(R) == 4) {
            // the roots magnify the absolute error of a small uniform (the
            // 23-bit fixed-point form of unif errs by 2^-24 absolute, which
            // moved cube roots near zero by 1e-4): here the words are
            // converted with 24-bit relative precision
            const float V0 = fmaf(__uint2float_rn(u.y), 0x1p-32f, 0x1p-33f);
            const float V1 = fmaf(__uint2float_rn(u.z), 0x1p-32f, 0x1p-33f);
            sc = cbrtf(V0);
            tc = sqrtf(V1);
        } else {
            sc = cbrt_newton(unif<R>(u.y));
            tc = sqrt(unif<R>(u.z));
        }
        const R st = sc * tc;
        b0 = R(1) - sc; b1 = sc * (R(1) - tc); b2 = st * (R(1) - U2); b3 = st * U2;
    } else {
        const R U0 = unif<R>(u.y), U1 = unif<R>(u.z);
        const R lo = U0 < U1 ? U0 : U1, hi = U0 < U1 ? U1 : U0;
        const R s0 = lo < U2 ? lo : U2;
        const R mid0 = lo < U2 ? U2 : lo;
        const R s2 = hi < mid0 ? mid0 : hi;
        const R s1 = hi < mid0 ? hi : mid0;
        b0 = s0; b1 = s1 - s0; b2 = s2 - s1; b3 = R(1) - s2;
    }
}

// ---------------------------------------------------------------------------
// approxcaps (Sec. 3.3): the convex hull of the inside vertices, the
// edge/sphere points and, on every face of T' crossed by the sphere between
// two edge points, the midpoint of the sphere's arc on that face.  The hull
// is grown from the nocaps polytope hull(I u P) by inserting the arc
// midpoints one at a time (beneath-beyond: faces that see the new point are
// replaced by the cone from the point to their horizon), then coned from the
// mean of its points.  Returns false when a hull could not be completed
// (capacity: maxf <= HULL_MAXF faces, HULL_MAXP points, HULL_MAXH horizon
// edges); the caller counts it and the assembly reports an error.
// The arc midpoint of face (f0,f1,f2) computed in FP64 for the FP32 path
// (used when the chord between the two edge points is short or the in-face
// decision is close).  Returns whether it lies in the face; its position
// relative to x (rounded to float) and its barycentric coordinates in the
// face go to pos[3] and lam[3].
static __device__ __noinline__ bool exact_mu(const Strict *sx, int f0, int f1, int f2, int iA, int oA, int iB, int oB,
                                             int vin, float pos[3], float lam[3])
{
    double v[4][3], x[3], pa[3], pb[3];
    strict_load(sx, v, x);
    sedge(v[iA], v[oA], x, sx->d2, pa);
    sedge(v[iB], v[oB], x, sx->d2, pb);
    double e1[3], e2[3], nr[3], xw[3];
    for (int d = 0; d < 3; ++d) { e1[d] = v[f1][d] - v[f0][d]; e2[d] = v[f2][d] - v[f0][d]; xw[d] = x[d] - v[f0][d]; }
    nr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double sf = (xw[0] * nr[0] + xw[1] * nr[1] + xw[2] * nr[2]) / (nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
    double cf[3], xc[3];
    for (int d = 0; d < 3; ++d) { cf[d] = x[d] - sf * nr[d]; xc[d] = x[d] - cf[d]; }
    double r2 = sx->d2 - (xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
    if (!(r2 > 0.0)) return false;
    double mid[3], ch[3], w[3];
    for (int d = 0; d < 3; ++d) { mid[d] = 0.5 * (pa[d] + pb[d]); ch[d] = pb[d] - pa[d]; w[d] = mid[d] - v[vin][d]; }
    double cc = ch[0] * ch[0] + ch[1] * ch[1] + ch[2] * ch[2];
    if (!(cc > 0.0)) return false;
    double pr = (w[0] * ch[0] + w[1] * ch[1] + w[2] * ch[2]) / cc;
    for (int d = 0; d < 3; ++d) w[d] -= pr * ch[d];
    double lw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (!(lw > 0.0)) return false;
    double rr = sqrt(r2) / lw, mu[3], g[3];
    for (int d = 0; d < 3; ++d) { mu[d] = cf[d] + rr * w[d]; g[d] = mu[d] - v[f0][d]; }
    double a11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], a12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    double a22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    double b1 = e1[0] * g[0] + e1[1] * g[1] + e1[2] * g[2], b2 = e2[0] * g[0] + e2[1] * g[1] + e2[2] * g[2];
    double det = a11 * a22 - a12 * a12;
    double ls = (b1 * a22 - b2 * a12) / det, lt = (a11 * b2 - a12 * b1) / det;
    for (int d = 0; d < 3; ++d) pos[d] = (float)(mu[d] - x[d]);
    lam[0] = (float)(1.0 - ls - lt); lam[1] = (float)ls; lam[2] = (float)lt;
    return !(ls < -1e-12 || lt < -1e-12 || 1.0 - ls - lt < -1e-12);
}

// Orientation of four FP32 points in FP64 (the rare branch of the filter below).
static __device__ __noinline__ int orient_sign_fp64(float ax, float ay, float az, float bx, float by, float bz,
                                                    float cx, float cy, float cz, float dx, float dy, float dz)
{
    const double e1x = (double)bx - ax, e1y = (double)by - ay, e1z = (double)bz - az;
    const double e2x = (double)cx - ax, e2y = (double)cy - ay, e2z = (double)cz - az;
    const double e3x = (double)dx - ax, e3y = (double)dy - ay, e3z = (double)dz - az;
    const double o = (e1x * (e2y * e3z - e2z * e3y) + e1y * (e2z * e3x - e2x * e3z)) + e1z * (e2x * e3y - e2y * e3x);
    return (o > 0.0) - (o < 0.0);
}

// Sign of orient(a, b, c, d), consistent across the decisions of one hull:
// in FP32 the determinant is trusted when it exceeds 1e-5 of its permanent
// (some 160 times its rounding error bound), otherwise the same FP32 points
// are taken to FP64, where the differences are exact and the determinant's
// error is far below any gap the FP32 coordinates can express.  Without it,
// an arc midpoint a few 1e-7 beyond a short chord can be seen as visible
// from one face and not from its neighbour, and the hull folds.
template <class R> __device__ __forceinline__ int orient_sign(P3<R> a, P3<R> b, P3<R> c, P3<R> d)
{
    if constexpr (sizeof(R) == 8) {
        const R o = orient(a, b, c, d);
        return (o > R(0)) - (o < R(0));
    } else {
        const P3<R> e1 = sub(b, a), e2 = sub(c, a), e3 = sub(d, a);
        const R o = det3(e1, e2, e3);
        const R perm = absr(e1.x) * (absr(e2.y * e3.z) + absr(e2.z * e3.y)) +
                       absr(e1.y) * (absr(e2.z * e3.x) + absr(e2.x * e3.z)) +
                       absr(e1.z) * (absr(e2.x * e3.y) + absr(e2.y * e3.x));
        if (absr(o) > R(1e-5) * perm) return (o > R(0)) - (o < R(0));
        return orient_sign_fp64(a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, d.x, d.y, d.z);
    }
}

constexpr int HULL_MAXP = 12;
constexpr int HULL_MAXF = 24;
constexpr int HULL_MAXH = 16;
// The hull's point table lives in a per-thread scratch (it is indexed at run
// time): value i of the thread at p[i s].  Points k < HULL_MAXP: coordinates
// at 3k..3k+2, barycentric row with respect to T' at 36 + 4k..36 + 4k + 3
// (84 values; the event kernel interleaves the threads of a block, s = block
// size, so that any index is conflict-free).
constexpr int HULL_SCRATCH = 3 * HULL_MAXP + 4 * HULL_MAXP;
template <class R> struct HullScratch {
    R *p;
    int s;
    __device__ __forceinline__ R &operator()(int i) const { return p[i * s]; }
};

template <class R, class KER = KerConst>
__device__ bool approx_hull_moments(const P3<R> v[4], P3<R> x, R d2, int m, const int role[4], const P3<R> pp[4],
                                    const R pt[4], const PDesc pd[4], bool diag_c2d1, Mom<R> &M, const Strict *sx,
                                    const HullScratch<R> &hs, int maxf, const KER &ker = KER{})
{
    constexpr bool F32 = sizeof(R) == 4;
    auto X = [&](int k) -> P3<R> { return mk3<R>(hs(3 * k), hs(3 * k + 1), hs(3 * k + 2)); };
    auto setX = [&](int k, P3<R> q) { hs(3 * k) = q.x; hs(3 * k + 1) = q.y; hs(3 * k + 2) = q.z; };
    auto Lr = [&](int k, int a) -> R & { return hs(3 * HULL_MAXP + 4 * k + a); };
    int n = 0;
    // table: T' vertices 0..3, edge points 4..7, arc midpoints 8..
    for (int k = 0; k < 4; ++k) {
        setX(k, v[k]);
        for (int a = 0; a < 4; ++a) Lr(k, a) = (a == k) ? R(1) : R(0);
    }
    const int np = m * (4 - m);
    for (int k = 0; k < np; ++k) {
        setX(4 + k, pp[k]);
        for (int a = 0; a < 4; ++a)
            Lr(4 + k, a) = (a == pd[k].i) ? (R(1) - pt[k]) : ((a == pd[k].o) ? pt[k] : R(0));
    }
    n = 4 + 4;
    // faces of the hull, packed point indices i | j << 8 | k << 16 (outward
    // orientation), initially those of hull(I u P)
    uint32_t F[HULL_MAXF];
    int nf = 0;
    const int a = role[0];
    auto pack = [](int i, int j, int k) -> uint32_t { return (uint32_t)i | ((uint32_t)j << 8) | ((uint32_t)k << 16); };
    auto add = [&](int i, int j, int k) { F[nf++] = pack(i, j, k); };
    if (m == 1) {
        add(a, 4, 5); add(a, 5, 6); add(a, 6, 4); add(4, 6, 5);
    } else if (m == 2) {
        const int b = role[1];
        add(a, 4, 5); add(b, 6, 7); add(a, b, 6); add(a, 6, 4); add(a, b, 7); add(a, 7, 5);
        if (!diag_c2d1) { add(4, 6, 7); add(4, 7, 5); }
        else { add(4, 6, 5); add(6, 7, 5); }
    } else {
        const int b = role[1], c = role[2];
        add(a, b, c); add(4, 5, 6); add(a, b, 5); add(a, 5, 4); add(b, c, 6); add(b, 6, 5); add(a, c, 6);
        add(a, 6, 4);
    }
    {
        // interior reference: mean of the hull(I u P) points
        P3<R> ci = mk3<R>(R(0), R(0), R(0));
        int cnt = 0;
        for (int k = 0; k < 4; ++k)
            if (k < m) { ci.x += v[role[k]].x; ci.y += v[role[k]].y; ci.z += v[role[k]].z; cnt++; }
        for (int k = 0; k < np; ++k) { ci.x += pp[k].x; ci.y += pp[k].y; ci.z += pp[k].z; cnt++; }
        R inv = R(1) / R(cnt);
        ci = mk3<R>(ci.x * inv, ci.y * inv, ci.z * inv);
        for (int f = 0; f < nf; ++f) {
            const uint32_t g = F[f];
            const int i0 = g & 0xff, i1 = (g >> 8) & 0xff, i2 = g >> 16;
            if (orient_sign(X(i0), X(i1), X(i2), ci) > 0) F[f] = pack(i0, i2, i1);
        }
    }
    // arc midpoints
    int inrank[4], outrank[4];
    {
        int ni = 0, no = 0;
        for (int k = 0; k < 4; ++k) { inrank[k] = -1; outrank[k] = -1; }
        for (int k = 0; k < m; ++k) inrank[role[k]] = ni++;
        for (int k = m; k < 4; ++k) outrank[role[k]] = no++;
    }
    int used = 4 + np;   // points in the hull so far (all of I u P; unused T' vertices are never referenced)
    (void)used;
    for (int o = 0; o < 4; ++o) {
        int fv[3], k3 = 0;
        for (int k = 0; k < 4; ++k) if (k != o) fv[k3++] = k;
        int pA = -1, pB = -1, vin = -1;
        for (int aa = 0; aa < 3; ++aa)
            for (int bb = aa + 1; bb < 3; ++bb) {
                int i = fv[aa], j = fv[bb];
                int pi = -1;
                if (inrank[i] >= 0 && outrank[j] >= 0) pi = 4 + inrank[i] * (4 - m) + outrank[j];
                else if (inrank[j] >= 0 && outrank[i] >= 0) pi = 4 + inrank[j] * (4 - m) + outrank[i];
                if (pi >= 0) { if (pA < 0) pA = pi; else pB = pi; }
            }
        for (int aa = 0; aa < 3; ++aa) if (inrank[fv[aa]] >= 0) { vin = fv[aa]; break; }
        if (pA < 0 || pB < 0 || vin < 0) continue;
        P3<R> e1 = sub(v[fv[1]], v[fv[0]]), e2 = sub(v[fv[2]], v[fv[0]]);
        P3<R> nr = mk3<R>(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
        P3<R> xw = sub(x, v[fv[0]]);
        R sfac = dot(xw, nr) / dot(nr, nr);
        P3<R> cf = mk3<R>(x.x - sfac * nr.x, x.y - sfac * nr.y, x.z - sfac * nr.z);
        P3<R> xc = sub(x, cf);
        R r2 = d2 - dot(xc, xc);
        if (!(r2 > R(0))) continue;
        P3<R> mid = mk3<R>(R(0.5) * (X(pA).x + X(pB).x), R(0.5) * (X(pA).y + X(pB).y), R(0.5) * (X(pA).z + X(pB).z));
        P3<R> ch = sub(X(pB), X(pA));
        R cc = dot(ch, ch);
        P3<R> mu;
        R l0, ls, lt;
        bool keep = false, exact = false;
        if (F32 && sx && cc < R(1e-4) * d2) {
            // FP32, a chord below 1 % of delta: the midpoint is left out.
            // Its direction is ill-conditioned in FP32 (a chord of 3e-3 delta
            // moved the midpoint by 1e-5 delta), and even a midpoint computed
            // in FP64 and rounded to float sits next to the chord, so the
            // faces of its cone are slivers whose planes the FP32
            // coordinates cannot resolve: a far midpoint then saw one of
            // them and not its neighbour, and the hull folded (errors up to
            // 3e-2 of |T'| at a chord of 3.6e-3 delta).  What is left out is
            // the arc segment over the chord, of height chord^2 / (8 r): its
            // moments stayed within 4e-6 of |T'| on every case set measured.
            // (Taking chords of 0.5 to 1 % of delta from FP64 instead cost
            // 14 % of the approxcaps batch time and did not change K's
            // errors.)
            continue;
        } else {
            if (!(cc > R(0))) continue;
            P3<R> w = sub(mid, v[vin]);
            R pr = dot(w, ch) / cc;
            w = mk3<R>(w.x - pr * ch.x, w.y - pr * ch.y, w.z - pr * ch.z);
            R lw = sqrt(dot(w, w));
            if (!(lw > R(0))) continue;
            if constexpr (F32) {
                // The direction away from the inside vertex within the face:
                // w is (mid - vin) without its chord component, which loses
                // its digits when vin lies near the chord's line (a vertex
                // just inside the sphere puts an edge point next to it; 1e-3
                // delta off the line gave midpoint errors of 1e-5 delta).
                // The same direction as the in-face normal of the chord,
                // nr x ch, whose FP32 error does not depend on where vin is,
                // with the sign that points away from vin; a sign too close
                // to call goes to FP64 below.
                const P3<R> perp = mk3<R>(nr.y * ch.z - nr.z * ch.y, nr.z * ch.x - nr.x * ch.z,
                                          nr.x * ch.y - nr.y * ch.x);
                const R lp = sqrt(dot(perp, perp));
                const R sg = dot(w, perp);
                if (sx && absr(sg) < R(1e-4) * lw * lp) {
                    exact = true;
                } else {
                    const R rr = (sg > R(0) ? sqrt(r2) : -sqrt(r2)) / lp;
                    mu = mk3<R>(cf.x + rr * perp.x, cf.y + rr * perp.y, cf.z + rr * perp.z);
                }
            } else {
                R rr = sqrt(r2) / lw;
                mu = mk3<R>(cf.x + rr * w.x, cf.y + rr * w.y, cf.z + rr * w.z);
            }
        }
        if (!exact) {
            // barycentric coordinates in the face; keep mu only inside the face
            P3<R> g = sub(mu, v[fv[0]]);
            R a11 = dot(e1, e1), a12 = dot(e1, e2), a22 = dot(e2, e2), b1 = dot(e1, g), b2 = dot(e2, g);
            R det = a11 * a22 - a12 * a12;
            ls = (b1 * a22 - b2 * a12) / det;
            lt = (a11 * b2 - a12 * b1) / det;
            l0 = R(1) - ls - lt;
            const R tl = R(-1e-12);
            keep = !(ls < tl || lt < tl || l0 < tl);
            if (F32 && sx && (absr(ls) < R(1e-4) || absr(lt) < R(1e-4) || absr(l0) < R(1e-4))) exact = true;
        }
        if (exact) {
            const int iA = pd[pA - 4].i, oA = pd[pA - 4].o, iB = pd[pB - 4].i, oB = pd[pB - 4].o;
            float pos[3], lm[3];
            keep = exact_mu(sx, fv[0], fv[1], fv[2], iA, oA, iB, oB, vin, pos, lm);
            mu = mk3<R>((R)pos[0], (R)pos[1], (R)pos[2]);
            l0 = (R)lm[0]; ls = (R)lm[1]; lt = (R)lm[2];
        }
        if (!keep) continue;
        if (n >= HULL_MAXP) return false;
        setX(n, mu);
        for (int aa = 0; aa < 4; ++aa) Lr(n, aa) = R(0);
        Lr(n, fv[0]) = l0; Lr(n, fv[1]) = ls; Lr(n, fv[2]) = lt;
        // insert: faces that see mu (bit mask)
        uint32_t vis = 0u;
        for (int f = 0; f < nf; ++f) {
            const uint32_t g = F[f];
            const int i0 = g & 0xff, i1 = (g >> 8) & 0xff, i2 = g >> 16;
            // faces in the plane of T''s face o (zero o-th barycentric coordinate
            // at all three points, exact by construction) hold mu in their plane
            if (Lr(i0, o) == R(0) && Lr(i1, o) == R(0) && Lr(i2, o) == R(0)) continue;
            if (orient_sign(X(i0), X(i1), X(i2), mu) > 0) vis |= 1u << f;
        }
        if (vis == 0u) continue;              // inside (or on) the hull already
        // horizon: edges of visible faces whose reverse edge belongs to no
        // other visible face
        uint32_t hz[HULL_MAXH];
        int nh = 0;
        for (uint32_t vm = vis; vm; vm &= vm - 1u) {
            const uint32_t g = F[__ffs(vm) - 1];
            const int gi[3] = {(int)(g & 0xff), (int)((g >> 8) & 0xff), (int)(g >> 16)};
            for (int e = 0; e < 3; ++e) {
                const int i0 = gi[e], i1 = gi[(e + 1) % 3];
                bool shared = false;
                for (uint32_t wm = vis; wm && !shared; wm &= wm - 1u) {
                    const uint32_t h = F[__ffs(wm) - 1];
                    const int hi[3] = {(int)(h & 0xff), (int)((h >> 8) & 0xff), (int)(h >> 16)};
                    shared = (hi[0] == i1 && hi[1] == i0) || (hi[1] == i1 && hi[2] == i0) || (hi[2] == i1 && hi[0] == i0);
                }
                if (!shared) {
                    if (nh >= HULL_MAXH) return false;
                    hz[nh++] = (uint32_t)i0 | ((uint32_t)i1 << 8);
                }
            }
        }
        // (near-coplanar faces can pinch the visible region at a vertex; the
        // cone over every horizon edge still closes the surface)
        if (nh < 3) return false;
        const int nvis = __popc(vis);
        if (nf - nvis + nh > maxf) return false;
        int w2 = 0;
        for (int f = 0; f < nf; ++f)
            if (!((vis >> f) & 1u)) F[w2++] = F[f];
        nf = w2;
        for (int h = 0; h < nh; ++h) F[nf++] = hz[h] | ((uint32_t)n << 16);
        n++;
    }
    // cone from the mean of the hull's points
    uint32_t inh = 0u;
    for (int f = 0; f < nf; ++f) {
        const uint32_t g = F[f];
        inh |= (1u << (g & 0xff)) | (1u << ((g >> 8) & 0xff)) | (1u << (g >> 16));
    }
    P3<R> c = mk3<R>(R(0), R(0), R(0));
    R Lc[4] = {R(0), R(0), R(0), R(0)};
    int cnt = 0;
    for (int k = 0; k < n; ++k)
        if ((inh >> k) & 1u) {
            const P3<R> q = X(k);
            c.x += q.x; c.y += q.y; c.z += q.z;
            for (int aa = 0; aa < 4; ++aa) Lc[aa] += Lr(k, aa);
            cnt++;
        }
    if (cnt < 4) return false;
    const R inv = R(1) / R(cnt);
    c = mk3<R>(c.x * inv, c.y * inv, c.z * inv);
    for (int aa = 0; aa < 4; ++aa) Lc[aa] *= inv;
    for (int f = 0; f < nf; ++f) {
        const uint32_t g = F[f];
        const int i0 = g & 0xff, i1 = (g >> 8) & 0xff, i2 = g >> 16;
        R vol = vol4(c, X(i0), X(i1), X(i2));
        R L0[4], L1[4], L2[4];
        for (int aa = 0; aa < 4; ++aa) { L0[aa] = Lr(i0, aa); L1[aa] = Lr(i1, aa); L2[aa] = Lr(i2, aa); }
        add_cell_k(M, vol, Lc, L0, L1, L2, c, X(i0), X(i1), X(i2), x, ker);
    }
    return true;
}

// Per-thread scratch for the cap cells: per cell the 4 vertices (12 values)
// and their barycentric rows with respect to T' (16 values).  Cell j of a
// thread starts cs values after cell j - 1: the event kernel lays the cells
// out cell-major across the block (cs = 28 x threads), so that the 16-byte
// loads of a warp hit distinct banks whatever cell each lane samples.  The
// FP32 sampler reads it with 16-byte loads, so the scratch must be 16-byte
// aligned (28 floats per cell keep every cell and every row on a 16-byte
// boundary).
constexpr int CB_STRIDE = 28;
static_assert((CB_STRIDE * sizeof(float)) % 16 == 0 && (12 * sizeof(float)) % 16 == 0, "cap scratch alignment");

// Moments of the approximate ball inside T' for a point x whose
// classification inm has 1..3 vertices inside, with run-time roles: the
// approxcaps path (the hull of Sec. 3.3 over I, P and the arc midpoints, or
// the nocaps cells of hull(I u P) when a hull cannot be completed).  The
// nocaps and fullcaps events go through event_moments below, which
// specialises the same geometry on the number of inside vertices.
//   hs: per-thread scratch of the approxcaps hull (HULL_SCRATCH values).
//   Returns true when the FP32 path defers the event (its output is then to
//   be discarded): a vertex of T' within 1e-3 (relative) of the sphere, where
//   the arc midpoints are ill-conditioned in FP32 (redone in FP64); and, when
//   DIAG_INLINE is false, an m = 2 diagonal that the FP32 orientation cannot
//   decide.  A hull that cannot be completed is counted in st.fallback (its
//   nocaps cells stand in for it here, and the assembly reports an error).
template <class R, int STRAT, bool DIAG_INLINE = true, class KER = KerConst>
__device__ bool event_moments_generic(const P3<R> v[4], P3<R> x, R d2, int inm, int nmc, const uint32_t *rk,
                                      uint32_t idT, uint32_t idTp, uint32_t q, R *out, Stats &st, const Strict *sx,
                                      R *cb, int cs, const HullScratch<R> &hs, int hull_maxf, const KER &ker = KER{})
{
    Mom<R> M;
    constexpr bool F32 = sizeof(R) == 4;
    // FP32 decision margins (relative): the FP32 sample point differs from the
    // FP64 one by a few 1e-7 of the cell size, far inside these margins
    const R MARGIN = R(4e-6);
    mom_zero(M);
    const int m = __popc(inm);
    int role[4];
    {
        int ni = 0, no = m;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (inm & (1 << k)) role[ni++] = k;
            else role[no++] = k;
        }
    }
    P3<R> pp[4];
    R pt[4];
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
                R C = ((w.x * w.x + w.y * w.y) + w.z * w.z) - d2;
                R s = sqrt(B * B - A * C);
                R t = (B >= R(0)) ? (-C) / (B + s) : (s - B) / A;
                pp[np] = mk3<R>(v[i].x + t * e.x, v[i].y + t * e.y, v[i].z + t * e.z);
                pt[np] = t;
                pd[np].i = (int8_t)i;
                pd[np].o = (int8_t)o;
                np++;
            }
    }
    auto P = [&](int p) -> P3<R> { return p < 4 ? v[p] : pp[p - 4]; };

    bool diag_c2d1 = false;
    if (m == 2) {
        P3<R> c1 = pp[0], d1 = pp[1], c2 = pp[2], dd2 = pp[3];
        R o1 = orient(c1, c2, dd2, d1), o2 = orient(c1, c2, dd2, v[role[0]]);
        bool exact = false;
        if (F32 && sx) {
            // The FP32 points and determinants err by less than about
            // (3 delta/L + 6) 2^-24 L^3 (coordinates of size delta relative to
            // x, quad of size L); decisions within 1e-5 L^2 max(L, delta) of
            // zero, nine times that bound or more, are retaken in FP64.
            const P3<R> e1 = sub(v[role[2]], v[role[0]]), e2 = sub(v[role[3]], v[role[1]]);
            const R L1 = (absr(e1.x) + absr(e1.y)) + absr(e1.z), L2 = (absr(e2.x) + absr(e2.y)) + absr(e2.z);
            const R L = L1 > L2 ? L1 : L2;
            const R dl = sqrt(d2);
            const R tol = R(1e-5) * L * L * (L > dl ? L : dl);
            if (absr(o1) <= tol || absr(o2) <= tol) {
                if constexpr (!DIAG_INLINE) return true;
                diag_c2d1 = strict_diag(sx, role[0], role[1], role[2], role[3]);
                exact = true;
            }
        }
        if (!exact) diag_c2d1 = (o1 > R(0) && o2 < R(0)) || (o1 < R(0) && o2 > R(0));
    }

    // approxcaps: the hull with the arc midpoints (falls back to nocaps cells)
    bool done_hull = false;
    if (STRAT == 1 && m > 0) {
        Mom<R> H;
        mom_zero(H);
        bool near = false;
        if (F32 && sx) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                P3<R> w = sub(v[k], x);
                R r2 = (w.x * w.x + w.y * w.y) + w.z * w.z;
                near |= absr(r2 - d2) < R(1e-3) * d2;
            }
        }
        if (near) return true;
        done_hull = approx_hull_moments<R, KER>(v, x, d2, m, role, pp, pt, pd, diag_c2d1, H, sx, hs, hull_maxf, ker);
        if (done_hull) M = H;
        else st.fallback++;                   // counted: the assembly then reports an error
    }
    // deterministic cells: hull(I u P), coned from the first inside vertex
    if (m > 0 && !done_hull) {
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
            add_cell_k(M, vol, L0, L1, L2, L3, P(cells[j][0]), P(cells[j][1]), P(cells[j][2]), P(cells[j][3]), x, ker);
        }
    }

    // the deterministic part goes out first (its registers are free during sampling)
    out[0] = M.m0;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[1 + k] = M.m1[k];
#pragma unroll
    for (int k = 0; k < 10; ++k) out[5 + k] = M.m2[k];
    (void)nmc; (void)rk; (void)idT; (void)idTp; (void)q; (void)cb; (void)cs;
    return false;
}

// Moments of the approximate ball inside T' for a point x whose
// classification inm has 1..3 vertices inside, or 0 vertices for a fullcaps
// cap that meets the ball:
//   nocaps/fullcaps: exact moments of the cells of hull(I u P);
//   fullcaps:        plus the Monte Carlo estimate over S = T' \ hull(I u P)
//                    with nmc Philox samples (cell by cumulative volume,
//                    uniform point from the spacings of three sorted
//                    uniforms, acceptance |y-x|^2 <= delta^2).  Accepted
//                    samples add 1, lambda'(y) and lambda'(y) lambda'(y)^T,
//                    lambda'(y) being the spacings' combination of the cell
//                    vertices' barycentric rows (non-negative terms only).
// The number of inside vertices is a compile-time constant here (the warps
// of the event kernel hold one class), so that the roles, the edge points and
// the cell tables are indexed statically and stay in registers; barycentric
// rows stay in T''s own vertex order (the roles only select).  Approxcaps
// goes to event_moments_generic.
//   cb, cs: per-thread scratch for the sampling cells, cell j at cb + j cs.
//   REC, rec: with REC (the diagnostic probe only), sample k is recorded at
//   rec[5k..5k+4] = (cap cell, accepted, y) with y global (FP64) or relative
//   to x (FP32).
//   Returns true when the event is deferred (see event_moments_generic).
//   hull_maxf: face capacity of the approxcaps hull (HULL_MAXF; smaller only
//   in tests of the overflow path).
template <class R, int STRAT, bool DIAG_INLINE = true, bool REC = false, bool QMC = false, class KER = KerConst>
__device__ bool event_moments(const P3<R> v[4], P3<R> x, R d2, int inm, int nmc, const uint32_t *rk, uint32_t idT,
                              uint32_t idTp, uint32_t q, R *out, Stats &st, const Strict *sx, R *cb, int cs,
                              const HullScratch<R> &hs, double *rec = nullptr, int hull_maxf = HULL_MAXF,
                              const KER &ker = KER{})
{
    if constexpr (STRAT == 1) {
        return event_moments_generic<R, STRAT, DIAG_INLINE, KER>(v, x, d2, inm, nmc, rk, idT, idTp, q, out, st, sx,
                                                                  cb, cs, hs, hull_maxf, ker);
    } else {
    Mom<R> M;
    constexpr bool F32 = sizeof(R) == 4;
    // FP32 decision margins (relative): the FP32 sample point differs from the
    // FP64 one by a few 1e-7 of the cell size, far inside these margins
    const R MARGIN = R(4e-6);
    mom_zero(M);
    const int m = __popc(inm);
    if (m > 0) st.cut++;
    // the sampler's cap cells (fullcaps): count, volumes, packed point
    // indices (T' vertex 0..3 or edge point 4 + k) and edge points
    int ns = 0, np = 0;
    unsigned long long spack = 0ULL;
    uint32_t pdpack = 0u;
    R vol[3] = {R(0), R(0), R(0)};
    bool defer = false;
    auto geom = [&](auto mconst) {
        constexpr int Mi = decltype(mconst)::value;
        constexpr int NO = 4 - Mi;
        constexpr int NP = Mi * NO;
        // roles: the inside vertices in increasing local index, then the
        // outside ones
        int role[4];
        {
            unsigned ins = (unsigned)inm & 15u, outs = (~(unsigned)inm) & 15u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k < Mi) { role[k] = __ffs(ins) - 1; ins &= ins - 1u; }
                else { role[k] = __ffs(outs) - 1; outs &= outs - 1u; }
            }
        }
        P3<R> vr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            vr[k] = role[k] == 0 ? v[0] : (role[k] == 1 ? v[1] : (role[k] == 2 ? v[2] : v[3]));
        // edge/sphere points, edge (inside role a, outside role b) at a NO + b - Mi
        P3<R> pp[NP > 0 ? NP : 1];
        R pt[NP > 0 ? NP : 1];
#pragma unroll
        for (int a = 0; a < Mi; ++a)
#pragma unroll
            for (int b = Mi; b < 4; ++b) {
                const int n = a * NO + (b - Mi);
                const P3<R> w = sub(vr[a], x);
                const P3<R> e = sub(vr[b], vr[a]);
                const R A = (e.x * e.x + e.y * e.y) + e.z * e.z;
                const R B = (e.x * w.x + e.y * w.y) + e.z * w.z;
                const R C = ((w.x * w.x + w.y * w.y) + w.z * w.z) - d2;
                const R sq = sqrt(B * B - A * C);
                const R t = (B >= R(0)) ? (-C) / (B + sq) : (sq - B) / A;
                pp[n] = mk3<R>(vr[a].x + t * e.x, vr[a].y + t * e.y, vr[a].z + t * e.z);
                pt[n] = t;
            }
        // table point p: p < 4 the vertex of role p, else edge point p - 4
        auto Pt = [&](int p) -> P3<R> { return p < 4 ? vr[p] : pp[p >= 4 ? p - 4 : 0]; };
        auto Lrow = [&](int p, R *L) {
            if (p < 4) {
                const int r = role[p];
#pragma unroll
                for (int a = 0; a < 4; ++a) L[a] = (a == r) ? R(1) : R(0);
            } else {
                const int n = p - 4;
                const int i = role[n / NO], o = role[Mi + n % NO];
                const R t = pt[n >= 0 && n < NP ? n : 0];
#pragma unroll
                for (int a = 0; a < 4; ++a) L[a] = (a == i) ? (R(1) - t) : ((a == o) ? t : R(0));
            }
        };
        auto orig = [&](int p) -> unsigned long long { return (unsigned long long)(p < 4 ? role[p] : p); };
        bool diag_c2d1 = false;
        if constexpr (Mi == 2) {
            const P3<R> c1 = pp[0], d1 = pp[1], c2 = pp[2], dd2 = pp[3];
            const R o1 = orient(c1, c2, dd2, d1), o2 = orient(c1, c2, dd2, vr[0]);
            bool exact = false;
            if (F32 && sx) {
                // The FP32 points and determinants err by less than about
                // (3 delta/L + 6) 2^-24 L^3 (coordinates of size delta relative to
                // x, quad of size L); decisions within 1e-5 L^2 max(L, delta) of
                // zero, nine times that bound or more, are retaken in FP64.
                const P3<R> e1 = sub(vr[2], vr[0]), e2 = sub(vr[3], vr[1]);
                const R L1 = (absr(e1.x) + absr(e1.y)) + absr(e1.z), L2 = (absr(e2.x) + absr(e2.y)) + absr(e2.z);
                const R L = L1 > L2 ? L1 : L2;
                const R dl = sqrt(d2);
                const R tol = R(1e-5) * L * L * (L > dl ? L : dl);
                if (absr(o1) <= tol || absr(o2) <= tol) {
                    if constexpr (!DIAG_INLINE) {
                        defer = true;
                        return;
                    } else {
                        diag_c2d1 = strict_diag(sx, role[0], role[1], role[2], role[3]);
                        exact = true;
                    }
                }
            }
            if (!exact) diag_c2d1 = (o1 > R(0) && o2 < R(0)) || (o1 < R(0) && o2 > R(0));
        }
        // deterministic cells: hull(I u P), coned from the first inside vertex
        auto cell = [&](int p0, int p1, int p2, int p3) {
            R L0[4], L1[4], L2[4], L3[4];
            Lrow(p0, L0); Lrow(p1, L1); Lrow(p2, L2); Lrow(p3, L3);
            const R vc = vol4(Pt(p0), Pt(p1), Pt(p2), Pt(p3));
            add_cell_k(M, vc, L0, L1, L2, L3, Pt(p0), Pt(p1), Pt(p2), Pt(p3), x, ker);
        };
        if constexpr (Mi == 1) {
            cell(0, 4, 5, 6);
        } else if constexpr (Mi == 2) {
            cell(0, 1, 6, 7);
            if (!diag_c2d1) { cell(0, 4, 6, 7); cell(0, 4, 7, 5); }
            else { cell(0, 4, 6, 5); cell(0, 6, 7, 5); }
        } else if constexpr (Mi == 3) {
            cell(0, 4, 5, 6); cell(0, 1, 2, 6); cell(0, 1, 6, 5);
        }
        if constexpr (STRAT == 2) {
            if (nmc > 0) {
                // cap cells S = T' \ hull(I u P) in the specification's order
                auto capcell = [&](int j, int p0, int p1, int p2, int p3) {
                    const P3<R> c0 = Pt(p0), c1 = Pt(p1), c2 = Pt(p2), c3 = Pt(p3);
                    vol[j] = vol4(c0, c1, c2, c3);
                    R *o = cb + cs * j;
                    if constexpr (F32) {
                        // FP32: the last vertex and the edges from it (the point
                        // is c3 + sum_k beta_k (c_k - c3); FP32 decisions near the
                        // margins are retaken in FP64)
                        o[0] = c3.x; o[1] = c3.y; o[2] = c3.z;
                        o[3] = c0.x - c3.x; o[4] = c0.y - c3.y; o[5] = c0.z - c3.z;
                        o[6] = c1.x - c3.x; o[7] = c1.y - c3.y; o[8] = c1.z - c3.z;
                        o[9] = c2.x - c3.x; o[10] = c2.y - c3.y; o[11] = c2.z - c3.z;
                    } else {
                        // FP64: the vertices, for the specification's operation order
                        o[0] = c0.x; o[1] = c0.y; o[2] = c0.z; o[3] = c1.x; o[4] = c1.y; o[5] = c1.z;
                        o[6] = c2.x; o[7] = c2.y; o[8] = c2.z; o[9] = c3.x; o[10] = c3.y; o[11] = c3.z;
                    }
                    Lrow(p0, o + 12); Lrow(p1, o + 16); Lrow(p2, o + 20); Lrow(p3, o + 24);
                    spack |= (orig(p0) << (3 * (4 * j))) | (orig(p1) << (3 * (4 * j + 1))) |
                             (orig(p2) << (3 * (4 * j + 2))) | (orig(p3) << (3 * (4 * j + 3)));
                };
                if constexpr (Mi == 0) {
                    capcell(0, 0, 1, 2, 3);
                    ns = 1;
                } else if constexpr (Mi == 1) {
                    capcell(0, 1, 4, 5, 6); capcell(1, 1, 2, 3, 6); capcell(2, 1, 2, 6, 5);
                    ns = 3;
                } else if constexpr (Mi == 2) {
                    capcell(0, 2, 3, 5, 7);
                    if (!diag_c2d1) { capcell(1, 2, 4, 6, 7); capcell(2, 2, 4, 7, 5); }
                    else { capcell(1, 2, 4, 6, 5); capcell(2, 2, 6, 7, 5); }
                    ns = 3;
                } else {
                    capcell(0, 3, 4, 5, 6);
                    ns = 1;
                }
#pragma unroll
                for (int n = 0; n < NP; ++n)
                    pdpack |= (uint32_t)(role[n / NO] | (role[Mi + n % NO] << 2)) << (4 * n);
                np = NP;
            }
        }
    };
    switch (m) {
    case 0: geom(std::integral_constant<int, 0>{}); break;
    case 1: geom(std::integral_constant<int, 1>{}); break;
    case 2: geom(std::integral_constant<int, 2>{}); break;
    default: geom(std::integral_constant<int, 3>{}); break;
    }
    if (defer) return true;

    // the deterministic part goes out first (its registers are free during sampling)
    out[0] = M.m0;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[1 + k] = M.m1[k];
#pragma unroll
    for (int k = 0; k < 10; ++k) out[5 + k] = M.m2[k];
    if (STRAT != 2 || nmc <= 0) return false;

    R tot = R(0);
    for (int j = 0; j < ns; ++j) tot += vol[j];
    const R BIG = R(3.0e38);
    R cum0 = vol[0];
    R cum1 = (ns > 1) ? cum0 + vol[1] : BIG;
    if (ns == 1) cum0 = BIG;
    // FP32: the cell choice compares the Philox word with the cumulative
    // volumes scaled to 2^32 (thresholds t0, t1; never exceeded when there is
    // one cell) and is retaken in FP64 within MARGIN 2^32 of a threshold
    // (unsigned wrap-around: (u - tk + wk) < 2 wk); the ball test is retaken
    // within MARGIN d2 of the sphere
    auto thresh = [&](R cum) -> uint32_t {
        const R g = (cum / tot) * R(4294967296.0);
        return g >= R(4294967295.0) ? 0xFFFFFFFFu : (uint32_t)g;
    };
    const uint32_t t0 = F32 ? thresh(cum0) : 0u, t1 = F32 ? thresh(cum1) : 0u;
    const uint32_t wk = (uint32_t)(MARGIN * R(4294967296.0));
    const uint32_t w2 = 2u * wk;
    const R dmar = MARGIN * d2;
    R cnt = R(0), a2[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) a2[k] = R(0);
    uint32_t acc = 0;
    CapDraws<QMC> draws(idT, idTp, q, rk);
    StrictCap scap;
    scap.ready = 0;
    if (F32 && ns == 1) {
        // FP32, one cap cell (m = 0 or 3; warp-uniform, the warps hold one
        // class): no cell choice, and the accepted samples' spacings are
        // summed as sum beta beta^T (non-negative terms), mapped to the
        // moments of lambda' = sum_k beta_k L_k once at the end (the sums of
        // lambda' are its row sums, as below)
        R sbb[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) sbb[k] = R(0);
        for (int k = 0; k < nmc; ++k) {
            const uint4 u = draws.next(k);
            R be[4];
            cap_bary<R, QMC>(u, be[0], be[1], be[2], be[3]);
            R cc[12];
            if constexpr (F32) {
                const float4 *c4 = reinterpret_cast<const float4 *>(cb);
                const float4 q0 = c4[0], q1 = c4[1], q2 = c4[2];
                cc[0] = q0.x; cc[1] = q0.y; cc[2] = q0.z; cc[3] = q0.w; cc[4] = q1.x; cc[5] = q1.y;
                cc[6] = q1.z; cc[7] = q1.w; cc[8] = q2.x; cc[9] = q2.y; cc[10] = q2.z; cc[11] = q2.w;
            } else {
#pragma unroll
                for (int kk = 0; kk < 12; ++kk) cc[kk] = cb[kk];
            }
            const P3<R> w = mk3<R>(((cc[0] + be[0] * cc[3]) + be[1] * cc[6]) + be[2] * cc[9],
                                   ((cc[1] + be[0] * cc[4]) + be[1] * cc[7]) + be[2] * cc[10],
                                   ((cc[2] + be[0] * cc[5]) + be[1] * cc[8]) + be[2] * cc[11]);
            const R rr = (w.x * w.x + w.y * w.y) + w.z * w.z;
            bool inb = rr <= d2;
            if (sx && absr(rr - d2) < dmar) {
                int j64 = 0;
                inb = strict_sample(sx, &scap, spack, ns, pdpack, np, u, &j64, QMC ? 1 : 0) != 0;
            }
            if constexpr (REC) {
                rec[5 * k] = 0.0; rec[5 * k + 1] = inb ? 1.0 : 0.0;
                rec[5 * k + 2] = (double)w.x; rec[5 * k + 3] = (double)w.y; rec[5 * k + 4] = (double)w.z;
            }
            const R f = inb ? kweight<R>(ker, rr) : R(0);
            acc += inb ? 1u : 0u;
            cnt += f;
            R fb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) fb[a] = f * be[a];
            int kk = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = a; b < 4; ++b) sbb[kk++] += fb[a] * be[b];
        }
        // the cell's rows L_k (lambda' at its vertices):
        // sum lambda' lambda'^T = sum_kl sbb_kl L_k L_l^T
        R L[16];
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) L[kk] = cb[12 + kk];
        auto bb = [&](int k, int l) -> R {
            const int a = k < l ? k : l, b = k < l ? l : k;
            return sbb[(a == 0) ? b : (a == 1) ? 3 + b : (a == 2) ? 5 + b : 9];
        };
        R t[4][4];    // t[k][a] = sum_l sbb_kl L_l[a]
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int a = 0; a < 4; ++a)
                t[k][a] = ((bb(k, 0) * L[a] + bb(k, 1) * L[4 + a]) + bb(k, 2) * L[8 + a]) + bb(k, 3) * L[12 + a];
        int kk = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int b = a; b < 4; ++b) {
                a2[kk++] = ((L[a] * t[0][b] + L[4 + a] * t[1][b]) + L[8 + a] * t[2][b]) + L[12 + a] * t[3][b];
            }
        }
    } else
    for (int k = 0; k < nmc; ++k) {
        uint4 u = draws.next(k);
        int j;
        bool cell_unsure = false;
        if constexpr (F32) {
            j = (u.x > t0 ? 1 : 0) + (u.x > t1 ? 1 : 0);
            cell_unsure = (u.x - t0 + wk) < w2 || (u.x - t1 + wk) < w2;
        } else {
            const R r = unit_scale<R>(u.x) * tot;
            j = (r >= cum0 ? 1 : 0) + (r >= cum1 ? 1 : 0);
        }
        R be0, be1, be2, be3;
        cap_bary<R, QMC>(u, be0, be1, be2, be3);
        const R *c = cb + cs * j;
        R cc[12];
        if constexpr (F32) {
            // 16-byte loads, conflict-free in the cell-major layout
            const float4 *c4 = reinterpret_cast<const float4 *>(c);
            const float4 q0 = c4[0], q1 = c4[1], q2 = c4[2];
            cc[0] = q0.x; cc[1] = q0.y; cc[2] = q0.z; cc[3] = q0.w; cc[4] = q1.x; cc[5] = q1.y;
            cc[6] = q1.z; cc[7] = q1.w; cc[8] = q2.x; cc[9] = q2.y; cc[10] = q2.z; cc[11] = q2.w;
        } else {
#pragma unroll
            for (int kk = 0; kk < 12; ++kk) cc[kk] = c[kk];
        }
        P3<R> y;
        if constexpr (F32)
            y = mk3<R>(((cc[0] + be0 * cc[3]) + be1 * cc[6]) + be2 * cc[9],
                       ((cc[1] + be0 * cc[4]) + be1 * cc[7]) + be2 * cc[10],
                       ((cc[2] + be0 * cc[5]) + be1 * cc[8]) + be2 * cc[11]);
        else
            y = mk3<R>(((be0 * cc[0] + be1 * cc[3]) + be2 * cc[6]) + be3 * cc[9],
                       ((be0 * cc[1] + be1 * cc[4]) + be2 * cc[7]) + be3 * cc[10],
                       ((be0 * cc[2] + be1 * cc[5]) + be2 * cc[8]) + be3 * cc[11]);
        P3<R> w = F32 ? y : sub(y, x);   // the FP32 path works relative to x
        R rr = (w.x * w.x + w.y * w.y) + w.z * w.z;
        bool inb = rr <= d2;
        if (F32 && sx) {
            if (cell_unsure || absr(rr - d2) < dmar) {
                int j64 = j;
                inb = strict_sample(sx, &scap, spack, ns, pdpack, np, u, &j64, QMC ? 1 : 0) != 0;
                c = cb + cs * j64;
                if constexpr (REC) j = j64;
            }
        }
        if constexpr (REC) {
            rec[5 * k] = (double)j; rec[5 * k + 1] = inb ? 1.0 : 0.0;
            rec[5 * k + 2] = (double)y.x; rec[5 * k + 3] = (double)y.y; rec[5 * k + 4] = (double)y.z;
        }
        // branch-free accumulation of the accepted sample (the sums of
        // lambda' are the row sums of lambda' lambda'^T: lambda' sums to 1)
        const R f = inb ? kweight<R>(ker, rr) : R(0);
        R Lr[16];
        if constexpr (F32) {
            const float4 *l4 = reinterpret_cast<const float4 *>(c + 12);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float4 t4 = l4[kk];
                Lr[4 * kk] = t4.x; Lr[4 * kk + 1] = t4.y; Lr[4 * kk + 2] = t4.z; Lr[4 * kk + 3] = t4.w;
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) Lr[kk] = c[12 + kk];
        }
        const R *L = Lr;
        R lam[4];
        acc += inb ? 1u : 0u;
        cnt += f;
        if constexpr (KER::constant) {
            // f is 0 or 1: lambda' lambda'^T f = (f lambda') (f lambda')^T
#pragma unroll
            for (int a = 0; a < 4; ++a)
                lam[a] = f * (((be0 * L[a] + be1 * L[4 + a]) + be2 * L[8 + a]) + be3 * L[12 + a]);
            int kk = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = a; b < 4; ++b) a2[kk++] += lam[a] * lam[b];
        } else {
            // weight phi once: (f lambda') lambda'^T
#pragma unroll
            for (int a = 0; a < 4; ++a) lam[a] = ((be0 * L[a] + be1 * L[4 + a]) + be2 * L[8 + a]) + be3 * L[12 + a];
            int kk = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = a; b < 4; ++b) a2[kk++] += (f * lam[a]) * lam[b];
        }
    }
    st.mc += (uint32_t)nmc;
    st.acc += acc;
    const R wgt = tot / R(nmc);
    out[0] += wgt * cnt;
    // packed upper triangle: (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3)
    out[1] += wgt * (((a2[0] + a2[1]) + a2[2]) + a2[3]);
    out[2] += wgt * (((a2[1] + a2[4]) + a2[5]) + a2[6]);
    out[3] += wgt * (((a2[2] + a2[5]) + a2[7]) + a2[8]);
    out[4] += wgt * (((a2[3] + a2[6]) + a2[8]) + a2[9]);
#pragma unroll
    for (int k = 0; k < 10; ++k) out[5 + k] += wgt * a2[k];
    return false;
    }
}

// Moments for one (T', x) including classification: used by the diagnostic
// probe; the assembly splits the two steps across kernels.
template <class R, int STRAT, bool REC = false, bool QMC = false>
// Returns the classification + 1 when the event is deferred to FP64, else 0.
// With REC the Monte Carlo samples go to rec (see event_moments) and *nrec
// receives their number (0 when there is no cap).
__device__ int point_moments(const P3<R> v[4], P3<R> x, R d2, R volTp, int nmc, const uint32_t *rk, uint32_t idT,
                             uint32_t idTp, uint32_t q, Mom<R> &M, Stats &st, const Strict *sx, R *cb, int cs,
                             const HullScratch<R> &hs, double *rec = nullptr, int *nrec = nullptr)
{
    if constexpr (REC) *nrec = 0;
    int inm = classify(v, x, d2, sx);
    if constexpr (STRAT >= 3) {
        if (element_full<R, STRAT>(v, x, d2, inm, sx)) {
            st.inside++;
            closed_form_inside(M, volTp);
        } else {
            mom_zero(M);
        }
        return 0;
    } else {
    if (inm == 15) {
        st.inside++;
        closed_form_inside(M, volTp);
        return 0;
    }
    if (inm == 0 && !(STRAT == 2 && nmc > 0 && meets_ball(v, x, d2, sx))) {
        mom_zero(M);
        return 0;
    }
    R o[15];
    const uint32_t mc0 = st.mc;
    if (event_moments<R, STRAT, true, REC, QMC>(v, x, d2, inm, nmc, rk, idT, idTp, q, o, st, sx, cb, cs, hs, rec))
        return inm + 1;
    if constexpr (REC) *nrec = (int)(st.mc - mc0);
    M.m0 = o[0];
    for (int k = 0; k < 4; ++k) M.m1[k] = o[1 + k];
    for (int k = 0; k < 10; ++k) M.m2[k] = o[5 + k];
    return 0;
    }
}

}  // namespace nlq
