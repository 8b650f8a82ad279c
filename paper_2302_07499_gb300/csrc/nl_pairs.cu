// Mesh upload and precompute, element-pair search on a uniform grid, and the
// fixed CSR pattern of the stiffness matrix.
//
// Compiled with -fmad=false: the quadrature points and the FP64 pair
// predicate follow a fixed operation order without fused multiply-add.
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "nl_internal.h"
#include "nl_quad.cuh"

namespace {

// 4-point degree-2 rule (Sec. 4.3.1): x_q = b*(v0+v1+v2+v3) + (a-b)*v_q with
// b = (5-sqrt5)/20 and a-b = sqrt5/5 (the doubles nearest those values).
__device__ __constant__ double kQB = 0x1.1b06d1d200913p-3;
__device__ __constant__ double kQAB = 0x1.c9f25c5bfedd9p-2;

__device__ __forceinline__ double3 ld3(const double4 v) { return make_double3(v.x, v.y, v.z); }
__device__ __forceinline__ double3 sub3(double3 a, double3 b) { return make_double3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double dot3(double3 a, double3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
__device__ __forceinline__ double det3(double3 a, double3 b, double3 c)
{
    return (a.x * (b.y * c.z - b.z * c.y) + a.y * (b.z * c.x - b.x * c.z)) + a.z * (b.x * c.y - b.y * c.x);
}
__device__ __forceinline__ float3 sub3f(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3f(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float det3f(float3 a, float3 b, float3 c)
{
    return a.x * (b.y * c.z - b.z * c.y) + a.y * (b.z * c.x - b.x * c.z) + a.z * (b.x * c.y - b.y * c.x);
}

// ordered-integer encoding of doubles for atomic min/max
__device__ __forceinline__ unsigned long long ord_enc(double x)
{
    unsigned long long u = __double_as_longlong(x);
    return (u & 0x8000000000000000ULL) ? ~u : (u | 0x8000000000000000ULL);
}
double ord_dec(unsigned long long u)
{
    unsigned long long v = (u & 0x8000000000000000ULL) ? (u & ~0x8000000000000000ULL) : ~u;
    double d;
    memcpy(&d, &v, sizeof(d));
    return d;
}

// ---------------------------------------------------------------------------
// mesh precompute
__global__ void k_mesh_prep(const double4 *__restrict__ verts, const int4 *__restrict__ tets, int64_t nv, int64_t nt,
                            double4 *tet_cr, double *tet_vol, int *err, unsigned long long *bb)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // bounding values as order-preserving integers; neutral for lanes past the
    // end or with a bad element
    unsigned long long enc[7] = {0ULL, ~0ULL, ~0ULL, ~0ULL, 0ULL, 0ULL, 0ULL};
    if (t < nt) {
        int4 e = tets[t];
        if (e.x < 0 || e.y < 0 || e.z < 0 || e.w < 0 || e.x >= nv || e.y >= nv || e.z >= nv || e.w >= nv) {
            atomicOr(err, 1);
            tet_cr[t] = make_double4(0, 0, 0, 0);
            tet_vol[t] = 0.0;
        } else {
            double3 v0 = ld3(verts[e.x]), v1 = ld3(verts[e.y]), v2 = ld3(verts[e.z]), v3 = ld3(verts[e.w]);
            double d = det3(sub3(v1, v0), sub3(v2, v0), sub3(v3, v0));
            if (!(d > 0.0)) atomicOr(err, 2);
            tet_vol[t] = fabs(d) / 6.0;
            double3 c = make_double3(0.25 * ((v0.x + v1.x) + (v2.x + v3.x)), 0.25 * ((v0.y + v1.y) + (v2.y + v3.y)),
                                     0.25 * ((v0.z + v1.z) + (v2.z + v3.z)));
            // the largest distance to a vertex: one square root of the
            // largest square (sqrt is monotone and correctly rounded)
            double r2 = dot3(sub3(v0, c), sub3(v0, c));
            r2 = fmax(r2, dot3(sub3(v1, c), sub3(v1, c)));
            r2 = fmax(r2, dot3(sub3(v2, c), sub3(v2, c)));
            r2 = fmax(r2, dot3(sub3(v3, c), sub3(v3, c)));
            const double r = sqrt(r2);
            tet_cr[t] = make_double4(c.x, c.y, c.z, r);
            enc[0] = ord_enc(r);
            enc[1] = ord_enc(c.x); enc[2] = ord_enc(c.y); enc[3] = ord_enc(c.z);
            enc[4] = enc[1]; enc[5] = enc[2]; enc[6] = enc[3];
        }
    }
    // warp reduction first: one atomic per warp and value
#pragma unroll
    for (int k = 0; k < 7; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, enc[k], o);
            enc[k] = (k >= 1 && k <= 3) ? (w < enc[k] ? w : enc[k]) : (w > enc[k] ? w : enc[k]);
        }
    if ((threadIdx.x & 31) == 0) {
        if (enc[0]) atomicMax(&bb[0], enc[0]);
        if (enc[1] != ~0ULL) { atomicMin(&bb[1], enc[1]); atomicMin(&bb[2], enc[2]); atomicMin(&bb[3], enc[3]); }
        if (enc[4]) { atomicMax(&bb[4], enc[4]); atomicMax(&bb[5], enc[5]); atomicMax(&bb[6], enc[6]); }
    }
}

__global__ void k_widen(const double *__restrict__ v3, double4 *v4, int64_t nv)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv) v4[i] = make_double4(v3[3 * i], v3[3 * i + 1], v3[3 * i + 2], 0.0);
}

__global__ void k_split_vol(const double *__restrict__ vol, float2 *hl, int64_t nt)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double v = vol[t];
    const float h = (float)v;
    hl[t] = make_float2(h, (float)(v - (double)h));
}

__global__ void k_split_coords(const double4 *__restrict__ verts, float4 *vhi, float4 *vlo, int64_t nv)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double4 v = verts[i];
    float hx = (float)v.x, hy = (float)v.y, hz = (float)v.z;
    vhi[i] = make_float4(hx, hy, hz, 0.f);
    vlo[i] = make_float4((float)(v.x - (double)hx), (float)(v.y - (double)hy), (float)(v.z - (double)hz), 0.f);
}

__global__ void k_flag_counts(const uint8_t *__restrict__ f, int64_t *cnt, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = f[i] ? 1 : 0;
}

__global__ void k_compact_flags(const uint8_t *__restrict__ f, const int64_t *__restrict__ off, int32_t *list,
                                int32_t *index_of, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (f[i]) {
        list[off[i]] = (int32_t)i;
        index_of[i] = (int32_t)off[i];
    } else {
        index_of[i] = -1;
    }
}

__global__ void k_quad_points(const double4 *__restrict__ verts, const int4 *__restrict__ tets,
                              const int32_t *__restrict__ outer_ids, int64_t n_outer, double *xq, float *xq_hl)
{
    int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_outer) return;
    int4 e = tets[outer_ids[o]];
    double4 v[4] = {verts[e.x], verts[e.y], verts[e.z], verts[e.w]};
    double s[3] = {(v[0].x + v[1].x) + (v[2].x + v[3].x), (v[0].y + v[1].y) + (v[2].y + v[3].y),
                   (v[0].z + v[1].z) + (v[2].z + v[3].z)};
    for (int q = 0; q < 4; ++q) {
        xq[12 * o + 3 * q + 0] = kQB * s[0] + kQAB * v[q].x;
        xq[12 * o + 3 * q + 1] = kQB * s[1] + kQAB * v[q].y;
        xq[12 * o + 3 * q + 2] = kQB * s[2] + kQAB * v[q].z;
        for (int d = 0; d < 3; ++d) {
            double x = xq[12 * o + 3 * q + d];
            float h = (float)x;
            xq_hl[24 * o + 6 * q + d] = h;
            xq_hl[24 * o + 6 * q + 3 + d] = (float)(x - (double)h);
        }
    }
}

__global__ void k_node_elem_count(const int4 *__restrict__ tets, int64_t nt, unsigned long long *cnt)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int4 e = tets[t];
    atomicAdd(&cnt[e.x], 1ULL); atomicAdd(&cnt[e.y], 1ULL);
    atomicAdd(&cnt[e.z], 1ULL); atomicAdd(&cnt[e.w], 1ULL);
}

__global__ void k_node_elem_fill(const int4 *__restrict__ tets, int64_t nt, unsigned long long *cursor, int32_t *ent)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int4 e = tets[t];
    int ids[4] = {e.x, e.y, e.z, e.w};
    for (int k = 0; k < 4; ++k) {
        unsigned long long p = atomicAdd(&cursor[ids[k]], 1ULL);
        ent[p] = (int32_t)((t << 2) | k);
    }
}

__global__ void k_max_seg(const int64_t *__restrict__ ptr, int64_t n, unsigned long long *mx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = (i < n) ? (unsigned long long)(ptr[i + 1] - ptr[i]) : 0ULL;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(mx, v);
}

// ---------------------------------------------------------------------------
// point-to-tetrahedron squared distance (closest point on each face the
// point lies outside of; zero when inside), FP64 and FP32 variants
__device__ double d2_point_tri(double3 p, double3 a, double3 b, double3 c)
{
    double3 ab = sub3(b, a), ac = sub3(c, a), ap = sub3(p, a);
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) return dot3(ap, ap);
    double3 bp = sub3(p, b);
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) return dot3(bp, bp);
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        double v = d1 / (d1 - d3);
        double3 q = make_double3(a.x + v * ab.x, a.y + v * ab.y, a.z + v * ab.z);
        double3 w = sub3(p, q);
        return dot3(w, w);
    }
    double3 cp = sub3(p, c);
    double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) return dot3(cp, cp);
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double w = d2 / (d2 - d6);
        double3 q = make_double3(a.x + w * ac.x, a.y + w * ac.y, a.z + w * ac.z);
        double3 r = sub3(p, q);
        return dot3(r, r);
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        double3 q = make_double3(b.x + w * (c.x - b.x), b.y + w * (c.y - b.y), b.z + w * (c.z - b.z));
        double3 r = sub3(p, q);
        return dot3(r, r);
    }
    double den = 1.0 / ((va + vb) + vc);
    double v = vb * den, w = vc * den;
    double3 q = make_double3((a.x + ab.x * v) + ac.x * w, (a.y + ab.y * v) + ac.y * w, (a.z + ab.z * v) + ac.z * w);
    double3 r = sub3(p, q);
    return dot3(r, r);
}

__device__ double d2_point_tet(double3 p, const double3 v[4])
{
    const int F[4][4] = {{1, 2, 3, 0}, {0, 2, 3, 1}, {0, 1, 3, 2}, {0, 1, 2, 3}};
    double best = 1e300;
    bool outside = false;
    for (int f = 0; f < 4; ++f) {
        double3 a = v[F[f][0]], b = v[F[f][1]], c = v[F[f][2]], o = v[F[f][3]];
        double sp = det3(sub3(b, a), sub3(c, a), sub3(p, a));
        double so = det3(sub3(b, a), sub3(c, a), sub3(o, a));
        if ((sp < 0.0 && so > 0.0) || (sp > 0.0 && so < 0.0)) {
            outside = true;
            best = fmin(best, d2_point_tri(p, a, b, c));
        }
    }
    return outside ? best : 0.0;
}

__device__ float d2_point_tri_f(float3 p, float3 a, float3 b, float3 c)
{
    float3 ab = sub3f(b, a), ac = sub3f(c, a), ap = sub3f(p, a);
    float d1 = dot3f(ab, ap), d2 = dot3f(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) return dot3f(ap, ap);
    float3 bp = sub3f(p, b);
    float d3 = dot3f(ab, bp), d4 = dot3f(ac, bp);
    if (d3 >= 0.f && d4 <= d3) return dot3f(bp, bp);
    float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
        float v = d1 / (d1 - d3);
        float3 w = make_float3(ap.x - v * ab.x, ap.y - v * ab.y, ap.z - v * ab.z);
        return dot3f(w, w);
    }
    float3 cp = sub3f(p, c);
    float d5 = dot3f(ab, cp), d6 = dot3f(ac, cp);
    if (d6 >= 0.f && d5 <= d6) return dot3f(cp, cp);
    float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        float w = d2 / (d2 - d6);
        float3 r = make_float3(ap.x - w * ac.x, ap.y - w * ac.y, ap.z - w * ac.z);
        return dot3f(r, r);
    }
    float va = d3 * d6 - d5 * d4;
    if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
        float w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        float3 r = make_float3(bp.x - w * (c.x - b.x), bp.y - w * (c.y - b.y), bp.z - w * (c.z - b.z));
        return dot3f(r, r);
    }
    float den = 1.f / (va + vb + vc);
    float v = vb * den, w = vc * den;
    float3 r = make_float3(ap.x - ab.x * v - ac.x * w, ap.y - ab.y * v - ac.y * w, ap.z - ab.z * v - ac.z * w);
    return dot3f(r, r);
}

__device__ float d2_point_tet_f(float3 p, const float3 v[4])
{
    const int F[4][4] = {{1, 2, 3, 0}, {0, 2, 3, 1}, {0, 1, 3, 2}, {0, 1, 2, 3}};
    float best = 3.0e38f;
    bool outside = false;
    for (int f = 0; f < 4; ++f) {
        float3 a = v[F[f][0]], b = v[F[f][1]], c = v[F[f][2]], o = v[F[f][3]];
        float sp = det3f(sub3f(b, a), sub3f(c, a), sub3f(p, a));
        float so = det3f(sub3f(b, a), sub3f(c, a), sub3f(o, a));
        if ((sp < 0.f && so > 0.f) || (sp > 0.f && so < 0.f)) {
            outside = true;
            best = fminf(best, d2_point_tri_f(p, a, b, c));
        }
    }
    return outside ? best : 0.f;
}

// ---------------------------------------------------------------------------
// uniform grid over element centroids
struct Grid {
    double lo[3];
    double cs;
    int n[3];
};

__global__ void k_cell_count(const double4 *__restrict__ tet_cr, int64_t nt, Grid g, int32_t *cell_of,
                             unsigned long long *cnt)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double4 c = tet_cr[t];
    int ix = (int)floor((c.x - g.lo[0]) / g.cs), iy = (int)floor((c.y - g.lo[1]) / g.cs),
        iz = (int)floor((c.z - g.lo[2]) / g.cs);
    ix = min(max(ix, 0), g.n[0] - 1); iy = min(max(iy, 0), g.n[1] - 1); iz = min(max(iz, 0), g.n[2] - 1);
    int cell = ix + g.n[0] * (iy + g.n[1] * iz);
    cell_of[t] = cell;
    atomicAdd(&cnt[cell], 1ULL);
}

__global__ void k_cell_fill(const int32_t *__restrict__ cell_of, int64_t nt, unsigned long long *cursor, int32_t *ent)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    unsigned long long p = atomicAdd(&cursor[cell_of[t]], 1ULL);
    ent[p] = (int32_t)t;
}

struct PairArgs {
    const double4 *verts;
    const float4 *vhi, *vlo;
    const int4 *tets;
    const double4 *tet_cr;
    const float4 *tet_cf;   // centroid and bounding radius in FP32 (conservative filters only)
    const int32_t *outer_ids;
    const double *xq;
    const int32_t *cell_of;
    const int64_t *cell_ptr;
    const int32_t *cell_ent;
    Grid g;
    int ks;                 // stencil radius in cells
    double delta, d2;
    float d2_lo, d2_hi;     // FP32 sure-accept / sure-reject bounds on d^2
    float qa_lo;            // sure-accept bound for distances from the hi parts alone (< 0: unused)
    float deltaf;
    int64_t n_outer;
};

// Conservative FP32 reach: a candidate is dropped only when its FP32 distance
// exceeds the exact limit by far more than the FP32 rounding of coordinates
// of magnitude <= 4 (relative 1e-5 plus 1e-5 absolute), so no pair of the
// exact predicate is ever lost.
__device__ __forceinline__ float reach_f(float lim) { return lim * 1.00001f + 1e-5f; }

__global__ void k_tet_cf(const double4 *__restrict__ cr, int64_t nt, float4 *cf)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) {
        double4 c = cr[t];
        cf[t] = make_float4((float)c.x, (float)c.y, (float)c.z, (float)c.w);
    }
}

// Exact predicate min_q d^2(x_q, T') <= delta^2, with an FP32 fast path on
// coordinates relative to x_q (double-float differences) and the FP64
// computation for every point whose FP32 distance is within the margin.
__device__ bool pair_predicate(const PairArgs &A, const double3 xq[4], const float3 xh[4], const float3 xl[4],
                               int4 e)
{
    int ids[4] = {e.x, e.y, e.z, e.w};
    float3 vh[4], vl[4];
    for (int k = 0; k < 4; ++k) {
        float4 h = A.vhi[ids[k]], l = A.vlo[ids[k]];
        vh[k] = make_float3(h.x, h.y, h.z);
        vl[k] = make_float3(l.x, l.y, l.z);
    }
    bool unsure[4];
    bool any_unsure = false;
    for (int q = 0; q < 4; ++q) {
        float3 w[4];
        float vmin = 3.0e38f;
        for (int k = 0; k < 4; ++k) {
            w[k] = make_float3((vh[k].x - xh[q].x) + (vl[k].x - xl[q].x), (vh[k].y - xh[q].y) + (vl[k].y - xl[q].y),
                               (vh[k].z - xh[q].z) + (vl[k].z - xl[q].z));
            vmin = fminf(vmin, dot3f(w[k], w[k]));
        }
        if (vmin < A.d2_lo) return true;                  // a vertex is surely within delta
        float d2 = (vmin <= A.d2_hi) ? vmin : d2_point_tet_f(make_float3(0.f, 0.f, 0.f), w);
        if (d2 < A.d2_lo) return true;
        unsure[q] = !(d2 > A.d2_hi);
        any_unsure |= unsure[q];
    }
    if (!any_unsure) return false;
    double3 v[4];
    for (int k = 0; k < 4; ++k) v[k] = ld3(A.verts[ids[k]]);
    for (int q = 0; q < 4; ++q)
        if (unsure[q] && d2_point_tet(xq[q], v) <= A.d2) return true;
    return false;
}

// Cheap part of the predicate: a vertex of T' surely within delta of an outer
// point (FP32 distance below the sure-accept bound).  Branch-free.
// The hi parts of the coordinates alone: their error (the lo parts, at most
// 2^-24 of the coordinates' magnitude, plus the rounding of the difference) is
// folded into qa_lo, set on the host from the mesh's extent.
__device__ bool quick_accept(const PairArgs &A, const float3 xh[4], int4 e)
{
    const int ids[4] = {e.x, e.y, e.z, e.w};
    float vmin = 3.0e38f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 h = A.vhi[ids[k]];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float3 w = make_float3(h.x - xh[q].x, h.y - xh[q].y, h.z - xh[q].z);
            vmin = fminf(vmin, dot3f(w, w));
        }
    }
    return vmin < A.qa_lo;
}

// One warp per outer element: scan the stencil of grid cells and test each
// candidate T'.  PASS 0 only bounds the number of candidates (centroid
// filter).  PASS 1 applies the cheap filters to 32 candidates at a time,
// queues the survivors per warp in shared memory, and runs the exact
// predicate on full warps of queued candidates: first the branch-free vertex
// test, then, on full warps of the candidates it leaves undecided (a second
// queue), the distance to T'.  The order of the output does not matter (every
// element's list is sorted afterwards); the survivors go to the outer
// element's bounded slot.
template <int PASS>
__global__ void __launch_bounds__(128, 4) k_pairs(PairArgs A, const int64_t *bptr, int64_t *counts, int32_t *out)
{
    __shared__ int32_t wq[4][64], wq2[4][64];
    int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (warp >= A.n_outer) return;
    int32_t *Q = wq[threadIdx.x >> 5], *Q2 = wq2[threadIdx.x >> 5];
    const unsigned lt = (1u << lane) - 1u;
    int32_t T = A.outer_ids[warp];
    const float4 cT = A.tet_cf[T];
    double3 xq[4];
    float3 xh[4], xl[4];
    if (PASS == 1) {
        for (int q = 0; q < 4; ++q) {
            xq[q] = make_double3(A.xq[12 * (int64_t)warp + 3 * q], A.xq[12 * (int64_t)warp + 3 * q + 1],
                                 A.xq[12 * (int64_t)warp + 3 * q + 2]);
            xh[q] = make_float3((float)xq[q].x, (float)xq[q].y, (float)xq[q].z);
            xl[q] = make_float3((float)(xq[q].x - (double)xh[q].x), (float)(xq[q].y - (double)xh[q].y),
                                (float)(xq[q].z - (double)xh[q].z));
        }
    }
    int cell = A.cell_of[T];
    int cx = cell % A.g.n[0], cy = (cell / A.g.n[0]) % A.g.n[1], cz = cell / (A.g.n[0] * A.g.n[1]);
    int64_t n = 0;
    int nq = 0, nq2 = 0;     // queued candidates (warp-uniform, below 64)
    int64_t base = (PASS == 1) ? bptr[warp] : 0;
    // full predicate on the last cnt candidates of the second queue (cnt <= 32)
    auto drain2 = [&](int cnt) {
        bool keep = false;
        int32_t Tp = -1;
        if (lane < cnt) {
            Tp = Q2[nq2 - cnt + lane];
            keep = pair_predicate(A, xq, xh, xl, A.tets[Tp]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) out[base + n + __popc(m & lt)] = Tp;
        n += __popc(m);
        nq2 -= cnt;
        __syncwarp();
    };
    // vertex test on the last cnt queued candidates (cnt <= 32): accepted ones
    // go out, undecided ones to the second queue
    auto drain = [&](int cnt) {
        bool keep = false, undecided = false;
        int32_t Tp = -1;
        if (lane < cnt) {
            Tp = Q[nq - cnt + lane];
            keep = quick_accept(A, xh, A.tets[Tp]);
            undecided = !keep;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) out[base + n + __popc(m & lt)] = Tp;
        n += __popc(m);
        nq -= cnt;
        const unsigned mu = __ballot_sync(0xffffffffu, undecided);
        if (undecided) Q2[nq2 + __popc(mu & lt)] = Tp;
        nq2 += __popc(mu);
        __syncwarp();
        if (nq2 >= 32) drain2(32);
    };
    for (int dz = -A.ks; dz <= A.ks; ++dz) {
        int z = cz + dz;
        if (z < 0 || z >= A.g.n[2]) continue;
        for (int dy = -A.ks; dy <= A.ks; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= A.g.n[1]) continue;
            for (int dx = -A.ks; dx <= A.ks; ++dx) {
                int x = cx + dx;
                if (x < 0 || x >= A.g.n[0]) continue;
                int c = x + A.g.n[0] * (y + A.g.n[1] * z);
                int64_t b = A.cell_ptr[c], e = A.cell_ptr[c + 1];
                for (int64_t s = b; s < e; s += 32) {
                    bool keep = false;
                    int32_t Tp = -1;
                    if (s + lane < e) {
                        Tp = A.cell_ent[s + lane];
                        const float4 cp = A.tet_cf[Tp];
                        const float ex = cT.x - cp.x, ey = cT.y - cp.y, ez = cT.z - cp.z;
                        const float lim = reach_f(A.deltaf + cT.w + cp.w);
                        keep = (ex * ex + ey * ey) + ez * ez <= lim * lim;
                        if (PASS == 1 && keep) {
                            // some outer point must reach the bounding ball of T'
                            const float lq = reach_f(A.deltaf + cp.w);
                            bool any = false;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float qx = xh[q].x - cp.x, qy = xh[q].y - cp.y, qz = xh[q].z - cp.z;
                                any |= (qx * qx + qy * qy) + qz * qz <= lq * lq;
                            }
                            keep = any;
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (PASS == 0) {
                        n += __popc(m);
                    } else {
                        if (keep) Q[nq + __popc(m & lt)] = Tp;
                        nq += __popc(m);
                        __syncwarp();
                        if (nq >= 32) drain(32);
                    }
                }
            }
        }
    }
    if (PASS == 1) {
        while (nq > 0) drain(nq < 32 ? nq : 32);
        while (nq2 > 0) drain2(nq2 < 32 ? nq2 : 32);
    }
    if (lane == 0) counts[warp] = n;
}

// Move each outer element's survivors from its bounded slot to the pair list.
__global__ void k_pairs_compact(const int64_t *__restrict__ bptr, const int64_t *__restrict__ ptr,
                                const int32_t *__restrict__ tmp, int64_t n_outer, int32_t *out)
{
    int64_t o = blockIdx.x;
    if (o >= n_outer) return;
    const int64_t b = bptr[o], p = ptr[o], n = ptr[o + 1] - ptr[o];
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) out[p + k] = tmp[b + k];
}

__global__ void k_pair_T(const int64_t *__restrict__ ptr, const int32_t *__restrict__ outer_ids, int64_t n_outer,
                         int32_t *pair_T)
{
    int64_t o = blockIdx.x;
    if (o >= n_outer) return;
    int32_t T = outer_ids[o];
    for (int64_t p = ptr[o] + threadIdx.x; p < ptr[o + 1]; p += blockDim.x) pair_T[p] = T;
}

__global__ void k_tp_count(const int32_t *__restrict__ tp, int64_t np, unsigned long long *cnt)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) atomicAdd(&cnt[tp[p]], 1ULL);
}

__global__ void k_tp_fill(const int32_t *__restrict__ tp, int64_t np, unsigned long long *cursor, int32_t *ent)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) {
        unsigned long long k = atomicAdd(&cursor[tp[p]], 1ULL);
        ent[k] = (int32_t)p;
    }
}

__global__ void k_u64_to_i64(const unsigned long long *a, int64_t *b, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int64_t)a[i];
}

// ---------------------------------------------------------------------------
// unique sorted gather with a shared-memory hash table (one block per group).
// The counting pass uses HCAP slots (up to UCAP unique keys); the filling pass
// knows the largest count and uses a table of twice that (rounded up to a
// power of two), so that it holds more blocks per SM.
constexpr int HCAP = 8192;      // hash slots of the counting pass
constexpr int UCAP = 4096;      // unique entries per group
constexpr int GB = 256;         // threads per block

__device__ __forceinline__ void hash_insert(int32_t *tab, int hcap, int *cnt, int *ovf, int32_t key)
{
    const unsigned mask = (unsigned)hcap - 1u;
    unsigned h = ((unsigned)key * 2654435761u) & mask;
    for (int probe = 0; probe < hcap; ++probe) {
        int32_t prev = atomicCAS(&tab[h], -1, key);
        if (prev == -1) { atomicAdd(cnt, 1); return; }
        if (prev == key) return;
        h = (h + 1) & mask;
    }
    atomicOr(ovf, 1);
}

__device__ void block_sort_write(int32_t *tab, int hcap, int32_t *list, int ucap, int *m, int32_t *dst)
{
    // compact the table, sort ascending, write out
    for (int i = threadIdx.x; i < hcap; i += blockDim.x) {
        int32_t k = tab[i];
        if (k != -1) {
            int p = atomicAdd(m, 1);
            if (p < ucap) list[p] = k;
        }
    }
    __syncthreads();
    int n = min(*m, ucap);
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int i = n + threadIdx.x; i < p2; i += blockDim.x) list[i] = 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    int32_t a = list[i], c = list[ixj];
                    bool up = ((i & k) == 0);
                    if ((a > c) == up) { list[i] = c; list[ixj] = a; }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = list[i];
}

struct NNArgs {
    const int4 *tets;
    const int32_t *outer_of;
    const int64_t *pair_ptr;
    const int32_t *pair_tp;
    const int32_t *pair_T;
    const int64_t *tp_ptr;
    const int32_t *tp_pair;
    int64_t nt;
};

__device__ __forceinline__ bool elem_active(const NNArgs &A, int64_t E)
{
    return A.outer_of[E] >= 0 || A.tp_ptr[E + 1] > A.tp_ptr[E];
}

// node set of all elements coupled with E (its partners, the outer elements
// that have E as a partner, and E itself)
template <int PASS>
__global__ void k_elem_nodes(NNArgs A, int hcap, int ucap, int64_t *cnt, const int64_t *ptr, int32_t *out, int *ovf)
{
    extern __shared__ int32_t sm[];
    int32_t *tab = sm;
    int32_t *list = sm + hcap;
    __shared__ int n_u, m_u;
    int64_t E = blockIdx.x;
    if (!elem_active(A, E)) {
        if (PASS == 0 && threadIdx.x == 0) cnt[E] = 0;
        return;
    }
    for (int i = threadIdx.x; i < hcap; i += blockDim.x) tab[i] = -1;
    if (threadIdx.x == 0) { n_u = 0; m_u = 0; }
    __syncthreads();
    if (threadIdx.x < 4) {
        int4 e = A.tets[E];
        int ids[4] = {e.x, e.y, e.z, e.w};
        hash_insert(tab, hcap, &n_u, ovf, ids[threadIdx.x]);
    }
    int32_t o = A.outer_of[E];
    if (o >= 0) {
        int64_t b = A.pair_ptr[o], e = A.pair_ptr[o + 1];
        for (int64_t i = b * 4 + threadIdx.x; i < e * 4; i += blockDim.x) {
            int4 t = A.tets[A.pair_tp[i >> 2]];
            int k = (int)(i & 3);
            hash_insert(tab, hcap, &n_u, ovf, k == 0 ? t.x : k == 1 ? t.y : k == 2 ? t.z : t.w);
        }
    }
    {
        int64_t b = A.tp_ptr[E], e = A.tp_ptr[E + 1];
        for (int64_t i = b * 4 + threadIdx.x; i < e * 4; i += blockDim.x) {
            int4 t = A.tets[A.pair_T[A.tp_pair[i >> 2]]];
            int k = (int)(i & 3);
            hash_insert(tab, hcap, &n_u, ovf, k == 0 ? t.x : k == 1 ? t.y : k == 2 ? t.z : t.w);
        }
    }
    __syncthreads();
    if (n_u > ucap) {
        if (threadIdx.x == 0) {
            atomicOr(ovf, 2);
            if (PASS == 0) cnt[E] = 0;
        }
        return;
    }
    if (PASS == 0) {
        if (threadIdx.x == 0) cnt[E] = n_u;
        return;
    }
    block_sort_write(tab, hcap, list, ucap, &m_u, out + ptr[E]);
}

// row of node r: union of the node sets of the active elements around r
template <int PASS>
__global__ void k_rows(NNArgs A, int hcap, int ucap, const int64_t *ne_ptr, const int32_t *ne_ent,
                       const int64_t *nn_ptr, const int32_t *nn_ent, int64_t *cnt, const int64_t *ptr, int32_t *out,
                       int *ovf)
{
    extern __shared__ int32_t sm[];
    int32_t *tab = sm;
    int32_t *list = sm + hcap;
    __shared__ int n_u, m_u;
    int64_t r = blockIdx.x;
    for (int i = threadIdx.x; i < hcap; i += blockDim.x) tab[i] = -1;
    if (threadIdx.x == 0) { n_u = 0; m_u = 0; }
    __syncthreads();
    for (int64_t k = ne_ptr[r]; k < ne_ptr[r + 1]; ++k) {
        int64_t E = ne_ent[k] >> 2;
        for (int64_t i = nn_ptr[E] + threadIdx.x; i < nn_ptr[E + 1]; i += blockDim.x)
            hash_insert(tab, hcap, &n_u, ovf, nn_ent[i]);
    }
    __syncthreads();
    if (n_u > ucap) {
        if (threadIdx.x == 0) {
            atomicOr(ovf, 2);
            if (PASS == 0) cnt[r] = 0;
        }
        return;
    }
    if (PASS == 0) {
        if (threadIdx.x == 0) cnt[r] = n_u;
        return;
    }
    block_sort_write(tab, hcap, list, ucap, &m_u, out + ptr[r]);
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int32_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_perm(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t nv, int32_t *perm,
                       int *bad)
{
    int64_t r = blockIdx.x;
    if (r >= nv) return;
    for (int64_t e = rowptr[r] + threadIdx.x; e < rowptr[r + 1]; e += blockDim.x) {
        int32_t c = col[e];
        int64_t b = rowptr[c], n = rowptr[c + 1] - b;
        int64_t k = lower_bound_i32(col + b, n, (int32_t)r);
        if (k >= n || col[b + k] != (int32_t)r) { atomicOr(bad, 4); perm[e] = (int32_t)e; }
        else perm[e] = (int32_t)(b + k);
    }
}

__global__ void k_elem_pos(NNArgs A, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                           int32_t *elem_pos, int *bad)
{
    int64_t E = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (E >= A.nt) return;
    if (!elem_active(A, E)) {
        for (int k = 0; k < 16; ++k) elem_pos[16 * E + k] = -1;
        return;
    }
    int4 e = A.tets[E];
    int ids[4] = {e.x, e.y, e.z, e.w};
    for (int i = 0; i < 4; ++i) {
        int64_t b = rowptr[ids[i]], n = rowptr[ids[i] + 1] - b;
        for (int j = 0; j < 4; ++j) {
            int64_t k = lower_bound_i32(col + b, n, ids[j]);
            if (k >= n || col[b + k] != ids[j]) { atomicOr(bad, 8); elem_pos[16 * E + 4 * i + j] = -1; }
            else elem_pos[16 * E + 4 * i + j] = (int32_t)(b + k);
        }
    }
}

__global__ void k_strip_len(const int4 *__restrict__ tets, const int32_t *__restrict__ outer_ids,
                            const int64_t *__restrict__ rowptr, int64_t n_outer, int64_t *len)
{
    int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_outer) return;
    int4 e = tets[outer_ids[o]];
    int ids[4] = {e.x, e.y, e.z, e.w};
    for (int i = 0; i < 4; ++i) len[4 * o + i] = rowptr[ids[i] + 1] - rowptr[ids[i]];
}

__global__ void k_row_len_max(const int64_t *__restrict__ rowptr, int64_t nv, unsigned long long *mx)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = (r < nv) ? (unsigned long long)(rowptr[r + 1] - rowptr[r]) : 0ULL;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(mx, v);
}

// Row views of K over the free rows: A = K[free, free] (COLLAR false; columns
// numbered among the free nodes) and L = K[free, collar] (COLLAR true; columns
// are node ids), each entry with its position in K.
template <bool COLLAR>
__global__ void k_a_count(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                          const int32_t *__restrict__ free_nodes, const int32_t *__restrict__ free_idx, int64_t n_free,
                          int64_t *cnt)
{
    int64_t fr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (fr >= n_free) return;
    int32_t r = free_nodes[fr];
    int64_t c = 0;
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) c += COLLAR ? (free_idx[col[e]] < 0) : (free_idx[col[e]] >= 0);
    cnt[fr] = c;
}

template <bool COLLAR>
__global__ void k_a_fill(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                         const int32_t *__restrict__ free_nodes, const int32_t *__restrict__ free_idx, int64_t n_free,
                         const int64_t *__restrict__ a_rowptr, int32_t *a_col, int32_t *a_src)
{
    int64_t fr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (fr >= n_free) return;
    int32_t r = free_nodes[fr];
    int64_t k = a_rowptr[fr];
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        const int32_t c = col[e];
        const int32_t f = free_idx[c];
        if (COLLAR ? f < 0 : f >= 0) { a_col[k] = COLLAR ? c : f; a_src[k] = (int32_t)e; ++k; }
    }
}

// A's rows padded to multiples of 4 entries: the lengths (in units of 4),
// then per row its columns and their positions in A, and the pads (column =
// the row itself, source -1)
__global__ void k_ap_len(const int64_t *__restrict__ a_rowptr, int64_t n, int64_t *len4)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) len4[r] = (a_rowptr[r + 1] - a_rowptr[r] + 3) / 4;
}

__global__ void k_ap_fill(const int64_t *__restrict__ a_rowptr, const int32_t *__restrict__ a_col, int64_t n,
                          const int64_t *__restrict__ rowptr4, int32_t *ap_col, int32_t *ap_src)
{
    int64_t r = blockIdx.x;
    if (r >= n) return;
    const int64_t b = a_rowptr[r], len = a_rowptr[r + 1] - b, o = 4 * rowptr4[r], lenp = 4 * (rowptr4[r + 1] - rowptr4[r]);
    for (int64_t k = threadIdx.x; k < lenp; k += blockDim.x) {
        const bool real = k < len;
        ap_col[o + k] = real ? a_col[b + k] : (int32_t)r;
        ap_src[o + k] = real ? (int32_t)(b + k) : -1;
    }
}

unsigned blocks_for(int64_t n, int threads) { return (unsigned)std::max<int64_t>(1, nl_cdiv<int64_t>(n, threads)); }

}  // namespace

// ===========================================================================
// ---------------------------------------------------------------------------
// Kuhn (Freudenthal) box mesh generated on the device: the same vertex and
// element numbering, coordinates and orientation as the host generator of
// the inputs module.  Vertex id = i + (n+1)(j + (n+1)k), coordinate lo + i*h
// with h = (hi - lo)/n; element id = 6*cell + p for the p-th axis permutation
// in lexicographic order, vertices (c, c+e_p1, c+e_p1+e_p2, c+(1,1,1)) with
// the last two swapped for the odd permutations (their signed volume is
// negative otherwise).  Omega = the cells inside [olo, ohi)^3 (grid
// indices); a node is free when strictly inside.
__global__ void k_box_verts(int n, double lo, double h, int olo, int ohi, double *v3, uint8_t *node_free)
{
    const int64_t m = n + 1;
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= m * m * m) return;
    const int i = (int)(id % m), j = (int)((id / m) % m), k = (int)(id / (m * m));
    v3[3 * id] = lo + (double)i * h;
    v3[3 * id + 1] = lo + (double)j * h;
    v3[3 * id + 2] = lo + (double)k * h;
    node_free[id] = (i > olo && i < ohi && j > olo && j < ohi && k > olo && k < ohi) ? 1 : 0;
}

__global__ void k_box_tets(int n, int olo, int ohi, int4 *tets, uint8_t *in_omega)
{
    const int64_t m = n + 1;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 6 * (int64_t)n * n * n) return;
    const int64_t cell = t / 6;
    const int p = (int)(t % 6);
    const int ci = (int)(cell % n), cj = (int)((cell / n) % n), ck = (int)(cell / ((int64_t)n * n));
    // lexicographic permutations of (0, 1, 2)
    const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int c[3] = {ci, cj, ck};
    int vid[4];
    for (int s = 0; s < 4; ++s) {
        if (s > 0) c[P[p][s - 1]] += 1;
        vid[s] = (int)(c[0] + m * (c[1] + m * c[2]));
    }
    const bool odd = (p == 1 || p == 2 || p == 5);
    tets[t] = odd ? make_int4(vid[0], vid[1], vid[3], vid[2]) : make_int4(vid[0], vid[1], vid[2], vid[3]);
    in_omega[t] = (ci >= olo && ci < ohi && cj >= olo && cj < ohi && ck >= olo && ck < ohi) ? 1 : 0;
}

// One parity class (i%2 + 2 (j%2) + 4 (k%2) == cls) of the jitter: vertex v
// moves by (2 U_d - 1) (jf h) along axis d, U_d = (w_d + 1/2) 2^-32 from the
// Philox4x32-10 words w of the counter (v, 0, 0, 0) under the key (k0, k1),
// unless it lies on a plane of the box or of Omega; the move is kept when
// every element holding v keeps a positive signed volume (the other three
// vertices at their current positions).  No two vertices of a class share an
// element, so the class is moved in one pass.
__global__ void k_box_jitter(int n, double lo, double h, int olo, int ohi, double jf, uint2 key, int cls, double *v3)
{
    const int64_t m = n + 1;
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= m * m * m) return;
    const int g[3] = {(int)(id % m), (int)((id / m) % m), (int)(id / (m * m))};
    if ((g[0] & 1) + 2 * (g[1] & 1) + 4 * (g[2] & 1) != cls) return;
    for (int d = 0; d < 3; ++d)
        if (g[d] == 0 || g[d] == n || g[d] == olo || g[d] == ohi) return;
    const uint4 w = nlq::philox4x32_10(make_uint4((uint32_t)id, 0u, 0u, 0u), key);
    const uint32_t wd[3] = {w.x, w.y, w.z};
    double trial[3];
    for (int d = 0; d < 3; ++d) {
        const double U = ((double)wd[d] + 0.5) * 0x1p-32;
        trial[d] = v3[3 * id + d] + (2.0 * U - 1.0) * (jf * h);
    }
    const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    bool ok = true;
    for (int cc = 0; cc < 8 && ok; ++cc) {
        const int cell[3] = {g[0] - (cc & 1), g[1] - ((cc >> 1) & 1), g[2] - ((cc >> 2) & 1)};
        if (cell[0] < 0 || cell[1] < 0 || cell[2] < 0 || cell[0] >= n || cell[1] >= n || cell[2] >= n) continue;
        for (int p = 0; p < 6 && ok; ++p) {
            int c[3] = {cell[0], cell[1], cell[2]};
            int64_t vid[4];
            for (int s = 0; s < 4; ++s) {
                if (s > 0) c[P[p][s - 1]] += 1;
                vid[s] = c[0] + m * (c[1] + m * (int64_t)c[2]);
            }
            if (p == 1 || p == 2 || p == 5) { const int64_t t = vid[2]; vid[2] = vid[3]; vid[3] = t; }
            if (vid[0] != id && vid[1] != id && vid[2] != id && vid[3] != id) continue;
            double q[4][3];
            for (int s = 0; s < 4; ++s)
                for (int d = 0; d < 3; ++d) q[s][d] = vid[s] == id ? trial[d] : v3[3 * vid[s] + d];
            double e1[3], e2[3], e3[3];
            for (int d = 0; d < 3; ++d) { e1[d] = q[1][d] - q[0][d]; e2[d] = q[2][d] - q[0][d]; e3[d] = q[3][d] - q[0][d]; }
            const double cx = e2[1] * e3[2] - e2[2] * e3[1];
            const double cy = e2[2] * e3[0] - e2[0] * e3[2];
            const double cz = e2[0] * e3[1] - e2[1] * e3[0];
            ok = ((e1[0] * cx + e1[1] * cy) + e1[2] * cz) > 0.0;
        }
    }
    if (ok)
        for (int d = 0; d < 3; ++d) v3[3 * id + d] = trial[d];
}

extern "C" nl_status nl_mesh_create_box(const nl_device *dev, double lo, double hi, int32_t cells, double omega_lo,
                                        double omega_hi, double jitter_frac, uint64_t seed, nl_mesh **out)
{
    nl_clear_error();
    if (!out) { nl_set_error("out is NULL"); return NL_EINVAL; }
    *out = nullptr;
    if (cells < 1 || cells > 1000 || !(hi > lo) || !isfinite(lo) || !isfinite(hi)) {
        nl_set_error("bad box (cells %d, [%g, %g])", cells, lo, hi);
        return NL_EINVAL;
    }
    const double h = (hi - lo) / cells;
    const double fo = (omega_lo - lo) / h, fe = (omega_hi - lo) / h;
    if (fabs(fo - nearbyint(fo)) > 1e-9 || fabs(fe - nearbyint(fe)) > 1e-9 || nearbyint(fo) < 0 ||
        nearbyint(fe) > cells || !(fe > fo)) {
        nl_set_error("Omega bounds must lie on grid planes inside the box");
        return NL_EINVAL;
    }
    if (!(jitter_frac >= 0.0 && jitter_frac < 0.5)) {
        nl_set_error("jitter_frac must lie in [0, 0.5)");
        return NL_EINVAL;
    }
    const int olo = (int)nearbyint(fo), ohi = (int)nearbyint(fe);
    const int64_t m = cells + 1, nv = m * m * m, nt = 6 * (int64_t)cells * cells * cells;
    DevArena tmp;
    if (dev) tmp.dev = *dev;
    nl_status st = NL_OK;
    try {
        cudaStream_t s = tmp.stream();
        double *v3 = tmp.get<double>(3 * nv);
        int4 *t4 = tmp.get<int4>(nt);
        uint8_t *om = tmp.get<uint8_t>(nt), *nf = tmp.get<uint8_t>(nv);
        { k_box_verts<<<blocks_for(nv, 256), 256, 0, s>>>(cells, lo, h, olo, ohi, v3, nf); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        if (jitter_frac > 0.0) {
            const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
            for (int cls = 0; cls < 8; ++cls) {
                { k_box_jitter<<<blocks_for(nv, 256), 256, 0, s>>>(cells, lo, h, olo, ohi, jitter_frac, key, cls, v3); nl_count_launch(); }
                NL_CHECK_LAUNCH();
            }
        }
        { k_box_tets<<<blocks_for(nt, 256), 256, 0, s>>>(cells, olo, ohi, t4, om); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        st = nl_mesh_create(dev, v3, nv, reinterpret_cast<const int32_t *>(t4), nt, om, nf, NL_DEVICE, out);
        NL_CUDA(cudaStreamSynchronize(s));
    } catch (NlError &e) {
        st = e.st;
    }
    tmp.release_all();
    return st;
}

extern "C" nl_status nl_mesh_create(const nl_device *dev, const double *verts, int64_t nv, const int32_t *tets,
                                    int64_t nt, const uint8_t *tet_in_omega, const uint8_t *node_free, int where,
                                    nl_mesh **out)
{
    nl_clear_error();
    if (!out) { nl_set_error("out is NULL"); return NL_EINVAL; }
    *out = nullptr;
    if (!verts || !tets || !tet_in_omega || !node_free) { nl_set_error("NULL input array"); return NL_EINVAL; }
    if (nv < 4 || nt < 1 || nv > 0x7fffffffLL || nt > (0x7fffffffLL >> 2)) {
        nl_set_error("bad sizes nv=%lld nt=%lld", (long long)nv, (long long)nt);
        return NL_EINVAL;
    }
    if (where != NL_HOST && where != NL_DEVICE) { nl_set_error("bad where"); return NL_EINVAL; }
    nl_mesh *m = new nl_mesh();
    if (dev) m->arena.dev = *dev;
    try {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            (void)cudaGetLastError();
            nl_set_error("no CUDA device available");
            throw NlError{NL_ECUDA};
        }
        cudaStream_t s = m->arena.stream();
        m->nv = nv;
        m->nt = nt;
        m->verts = m->arena.get<double4>(nv);
        m->tets = m->arena.get<int4>(nt);
        m->in_omega = m->arena.get<uint8_t>(nt);
        m->node_free = m->arena.get<uint8_t>(nv);
        Scratch sc(&m->arena);
        // coordinates arrive as [nv][3]; widen to double4 on the device
        double *v3 = sc.get<double>(3 * nv);
        cudaMemcpyKind kind = (where == NL_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        NL_CUDA(cudaMemcpyAsync(v3, verts, sizeof(double) * 3 * nv, kind, s));
        NL_CUDA(cudaMemcpyAsync(m->tets, tets, sizeof(int4) * nt, kind, s));
        NL_CUDA(cudaMemcpyAsync(m->in_omega, tet_in_omega, nt, kind, s));
        NL_CUDA(cudaMemcpyAsync(m->node_free, node_free, nv, kind, s));
        { k_widen<<<blocks_for(nv, 256), 256, 0, s>>>(v3, m->verts, nv); nl_count_launch(); }
        NL_CHECK_LAUNCH();

        m->tet_cr = m->arena.get<double4>(nt);
        m->tet_vol = m->arena.get<double>(nt);
        int *err = sc.get<int>(1);
        unsigned long long *bb = sc.get<unsigned long long>(8);
        NL_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        unsigned long long init[8];
        init[0] = 0ULL;
        for (int i = 1; i <= 3; ++i) init[i] = ~0ULL;
        for (int i = 4; i <= 6; ++i) init[i] = 0ULL;
        init[7] = 0ULL;
        NL_CUDA(cudaMemcpyAsync(bb, init, sizeof(init), cudaMemcpyHostToDevice, s));
        { k_mesh_prep<<<blocks_for(nt, 256), 256, 0, s>>>(m->verts, m->tets, nv, nt, m->tet_cr, m->tet_vol, err, bb); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        m->vhi = m->arena.get<float4>(nv);
        m->vlo = m->arena.get<float4>(nv);
        { k_split_coords<<<blocks_for(nv, 256), 256, 0, s>>>(m->verts, m->vhi, m->vlo, nv); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        m->vol_hl = m->arena.get<float2>(nt);
        { k_split_vol<<<blocks_for(nt, 256), 256, 0, s>>>(m->tet_vol, m->vol_hl, nt); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        int herr = 0;
        unsigned long long hbb[8];
        NL_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaMemcpyAsync(hbb, bb, sizeof(hbb), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        NL_REQUIRE(!(herr & 1), "a vertex id is out of range [0, %lld)", (long long)nv);
        NL_REQUIRE(!(herr & 2), "an element has non-positive signed volume (vertices must be positively oriented)");
        m->rmax = ord_dec(hbb[0]);
        for (int d = 0; d < 3; ++d) { m->bbmin[d] = ord_dec(hbb[1 + d]); m->bbmax[d] = ord_dec(hbb[4 + d]); }

        // outer elements and free nodes
        int64_t *cnt = sc.get<int64_t>(std::max(nt, nv) + 1);
        int64_t *off = sc.get<int64_t>(std::max(nt, nv) + 1);
        { k_flag_counts<<<blocks_for(nt, 256), 256, 0, s>>>(m->in_omega, cnt, nt); nl_count_launch(); }
        m->n_outer = nl_scan_counts(cnt, off, nt, &m->arena, s);
        NL_REQUIRE(m->n_outer > 0, "no element of Omega");
        m->outer_ids = m->arena.get<int32_t>(m->n_outer);
        m->outer_of = m->arena.get<int32_t>(nt);
        { k_compact_flags<<<blocks_for(nt, 256), 256, 0, s>>>(m->in_omega, off, m->outer_ids, m->outer_of, nt); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        { k_flag_counts<<<blocks_for(nv, 256), 256, 0, s>>>(m->node_free, cnt, nv); nl_count_launch(); }
        m->n_free = nl_scan_counts(cnt, off, nv, &m->arena, s);
        NL_REQUIRE(m->n_free > 0, "no free node");
        m->free_nodes = m->arena.get<int32_t>(m->n_free);
        m->free_idx = m->arena.get<int32_t>(nv);
        { k_compact_flags<<<blocks_for(nv, 256), 256, 0, s>>>(m->node_free, off, m->free_nodes, m->free_idx, nv); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        m->xq = m->arena.get<double>(12 * m->n_outer);
        m->xq_hl = m->arena.get<float>(24 * m->n_outer);
        { k_quad_points<<<blocks_for(m->n_outer, 128), 128, 0, s>>>(m->verts, m->tets, m->outer_ids, m->n_outer, m->xq, m->xq_hl); nl_count_launch(); }
        NL_CHECK_LAUNCH();

        // node -> incident elements, sorted by element id
        unsigned long long *ucnt = sc.get<unsigned long long>(nv);
        NL_CUDA(cudaMemsetAsync(ucnt, 0, sizeof(unsigned long long) * nv, s));
        { k_node_elem_count<<<blocks_for(nt, 256), 256, 0, s>>>(m->tets, nt, ucnt); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        { k_u64_to_i64<<<blocks_for(nv, 256), 256, 0, s>>>(ucnt, cnt, nv); nl_count_launch(); }
        m->ne_ptr = m->arena.get<int64_t>(nv + 1);
        int64_t ninc = nl_scan_counts(cnt, m->ne_ptr, nv, &m->arena, s);
        m->ne_ent = m->arena.get<int32_t>(ninc);
        { k_u64_to_i64<<<blocks_for(nv, 256), 256, 0, s>>>(ucnt, cnt, nv); nl_count_launch(); }
        NL_CUDA(cudaMemcpyAsync(ucnt, m->ne_ptr, sizeof(int64_t) * nv, cudaMemcpyDeviceToDevice, s));
        { k_node_elem_fill<<<blocks_for(nt, 256), 256, 0, s>>>(m->tets, nt, ucnt, m->ne_ent); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        unsigned long long *mx = sc.get<unsigned long long>(1);
        NL_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
        { k_max_seg<<<blocks_for(nv, 256), 256, 0, s>>>(m->ne_ptr, nv, mx); nl_count_launch(); }
        unsigned long long hmx = 0;
        NL_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        nl_segmented_sort_i32(m->ne_ent, m->ne_ptr, nv, (int64_t)hmx, &m->arena, s);
        NL_CUDA(cudaStreamSynchronize(s));
    } catch (NlError &e) {
        m->arena.release_all();
        delete m;
        return e.st;
    }
    *out = m;
    return NL_OK;
}

extern "C" void nl_mesh_destroy(nl_mesh *m)
{
    if (!m) return;
    m->arena.release_all();
    delete m;
}

// ===========================================================================
nl_status nl_pairs_build_impl(nl_mesh *m, double delta, nl_pairs **out)
{
    nl_pairs *P = new nl_pairs();
    P->arena.dev = m->arena.dev;
    P->mesh = m;
    P->delta = delta;
    try {
        cudaStream_t s = P->arena.stream();
        Scratch sc(&P->arena);
        const int64_t nt = m->nt, nv = m->nv, no = m->n_outer;

        // grid
        Grid g;
        const int ks = 2;
        g.cs = (delta + 2.0 * m->rmax) / ks;
        for (int d = 0; d < 3; ++d) {
            g.lo[d] = m->bbmin[d];
            double ext = m->bbmax[d] - m->bbmin[d];
            int64_t n = (int64_t)floor(ext / g.cs) + 1;
            g.n[d] = (int)std::max<int64_t>(1, std::min<int64_t>(n, 1024));
        }
        if ((double)g.n[0] * g.n[1] * g.n[2] > 3e7) {
            // very small delta relative to the box: coarsen the grid
            double f = cbrt((double)g.n[0] * g.n[1] * g.n[2] / 3e7) * 1.01;
            g.cs *= f;
            for (int d = 0; d < 3; ++d)
                g.n[d] = (int)std::max<int64_t>(1, (int64_t)floor((m->bbmax[d] - m->bbmin[d]) / g.cs) + 1);
        }
        int64_t ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
        int32_t *cell_of = sc.get<int32_t>(nt);
        unsigned long long *ucnt = sc.get<unsigned long long>(std::max(ncell, nt) + 1);
        int64_t *cnt = sc.get<int64_t>(std::max(std::max(ncell, nt), std::max(no, nv)) + 1);
        NL_CUDA(cudaMemsetAsync(ucnt, 0, sizeof(unsigned long long) * ncell, s));
        { k_cell_count<<<blocks_for(nt, 256), 256, 0, s>>>(m->tet_cr, nt, g, cell_of, ucnt); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        { k_u64_to_i64<<<blocks_for(ncell, 256), 256, 0, s>>>(ucnt, cnt, ncell); nl_count_launch(); }
        int64_t *cell_ptr = sc.get<int64_t>(ncell + 1);
        nl_scan_counts(cnt, cell_ptr, ncell, &P->arena, s);
        int32_t *cell_ent = sc.get<int32_t>(nt);
        NL_CUDA(cudaMemcpyAsync(ucnt, cell_ptr, sizeof(int64_t) * ncell, cudaMemcpyDeviceToDevice, s));
        { k_cell_fill<<<blocks_for(nt, 256), 256, 0, s>>>(cell_of, nt, ucnt, cell_ent); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        unsigned long long *mx = sc.get<unsigned long long>(1);
        unsigned long long hmx = 0;
        NL_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
        { k_max_seg<<<blocks_for(ncell, 256), 256, 0, s>>>(cell_ptr, ncell, mx); nl_count_launch(); }
        NL_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        nl_segmented_sort_i32(cell_ent, cell_ptr, ncell, (int64_t)hmx, &P->arena, s);

        // pairs
        PairArgs A;
        float4 *tet_cf = sc.get<float4>(nt);
        { k_tet_cf<<<blocks_for(nt, 256), 256, 0, s>>>(m->tet_cr, nt, tet_cf); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        A.verts = m->verts; A.vhi = m->vhi; A.vlo = m->vlo; A.tets = m->tets; A.tet_cr = m->tet_cr; A.tet_cf = tet_cf;
        A.outer_ids = m->outer_ids; A.xq = m->xq; A.cell_of = cell_of; A.cell_ptr = cell_ptr; A.cell_ent = cell_ent;
        A.g = g; A.ks = ks; A.delta = delta; A.d2 = delta * delta;
        A.d2_lo = (float)(A.d2 * (1.0 - 1e-4)); A.d2_hi = (float)(A.d2 * (1.0 + 1e-4));
        {
            // |coordinates| <= M: each component of a hi-part difference errs
            // by at most 3 M 2^-24, the vector by e = 3 sqrt(3) M 2^-24; a
            // squared FP32 distance below (delta - 2e)^2 (less a relative
            // 1e-6 for its own rounding) is then surely within delta
            double M = 0.0;
            for (int d = 0; d < 3; ++d)
                M = std::max(M, std::max(fabs(m->bbmin[d] - m->rmax), fabs(m->bbmax[d] + m->rmax)));
            const double e = 3.0 * sqrt(3.0) * M * 0x1p-24;
            const double r = delta - 2.0 * e;
            A.qa_lo = r > 0.0 ? (float)std::min(A.d2 * (1.0 - 1e-4), r * r * (1.0 - 1e-6)) : -1.0f;
        }
        A.deltaf = (float)delta;
        A.n_outer = no;
        unsigned pblocks = blocks_for(no * 32, 128);
        { k_pairs<0><<<pblocks, 128, 0, s>>>(A, nullptr, cnt, nullptr); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        int64_t *bptr = sc.get<int64_t>(no + 1);
        const int64_t nbound = nl_scan_counts(cnt, bptr, no, &P->arena, s);
        int32_t *tmp = sc.get<int32_t>(nbound);
        { k_pairs<1><<<pblocks, 128, 0, s>>>(A, bptr, cnt, tmp); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        P->pair_ptr = P->arena.get<int64_t>(no + 1);
        P->npairs = nl_scan_counts(cnt, P->pair_ptr, no, &P->arena, s);
        NL_REQUIRE(P->npairs < 0x7fffffffLL, "%lld pairs exceed the int32 pair index", (long long)P->npairs);
        P->pair_tp = P->arena.get<int32_t>(P->npairs);
        { k_pairs_compact<<<(unsigned)no, 128, 0, s>>>(bptr, P->pair_ptr, tmp, no, P->pair_tp); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        NL_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
        { k_max_seg<<<blocks_for(no, 256), 256, 0, s>>>(P->pair_ptr, no, mx); nl_count_launch(); }
        NL_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        P->max_pairs_per_outer = (int64_t)hmx;
        nl_segmented_sort_i32(P->pair_tp, P->pair_ptr, no, (int64_t)hmx, &P->arena, s);
        P->pair_T = P->arena.get<int32_t>(P->npairs);
        { k_pair_T<<<(unsigned)no, 128, 0, s>>>(P->pair_ptr, m->outer_ids, no, P->pair_T); nl_count_launch(); }
        NL_CHECK_LAUNCH();

        // transposed pair list: pairs by T', increasing pair id
        NL_CUDA(cudaMemsetAsync(ucnt, 0, sizeof(unsigned long long) * nt, s));
        { k_tp_count<<<blocks_for(P->npairs, 256), 256, 0, s>>>(P->pair_tp, P->npairs, ucnt); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        { k_u64_to_i64<<<blocks_for(nt, 256), 256, 0, s>>>(ucnt, cnt, nt); nl_count_launch(); }
        P->tp_ptr = P->arena.get<int64_t>(nt + 1);
        nl_scan_counts(cnt, P->tp_ptr, nt, &P->arena, s);
        P->tp_pair = P->arena.get<int32_t>(P->npairs);
        NL_CUDA(cudaMemcpyAsync(ucnt, P->tp_ptr, sizeof(int64_t) * nt, cudaMemcpyDeviceToDevice, s));
        { k_tp_fill<<<blocks_for(P->npairs, 256), 256, 0, s>>>(P->pair_tp, P->npairs, ucnt, P->tp_pair); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        NL_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
        { k_max_seg<<<blocks_for(nt, 256), 256, 0, s>>>(P->tp_ptr, nt, mx); nl_count_launch(); }
        NL_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        nl_segmented_sort_i32(P->tp_pair, P->tp_ptr, nt, (int64_t)hmx, &P->arena, s);

        // node sets per element, then rows
        NNArgs N;
        N.tets = m->tets; N.outer_of = m->outer_of; N.pair_ptr = P->pair_ptr; N.pair_tp = P->pair_tp;
        N.pair_T = P->pair_T; N.tp_ptr = P->tp_ptr; N.tp_pair = P->tp_pair; N.nt = nt;
        int *ovf = sc.get<int>(1);
        NL_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
        const size_t hsm = sizeof(int32_t) * (HCAP + UCAP);   // the largest table + list (both passes)
        NL_CUDA(cudaFuncSetAttribute(k_elem_nodes<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
        NL_CUDA(cudaFuncSetAttribute(k_elem_nodes<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
        NL_CUDA(cudaFuncSetAttribute(k_rows<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
        NL_CUDA(cudaFuncSetAttribute(k_rows<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
        const size_t hsm0 = sizeof(int32_t) * HCAP;             // counting pass: no list
        // the filling pass: a table of twice the largest count, a list of it
        auto check_overflow = [&]() {
            int hovf = 0;
            NL_CUDA(cudaMemcpyAsync(&hovf, ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
            NL_CUDA(cudaStreamSynchronize(s));
            NL_REQUIRE(hovf == 0, "sparsity pattern overflow (more than %d columns in a row); delta/h too large",
                       UCAP);
        };
        auto fill_shape = [&](const int64_t *ptr, int64_t n, int &hcap, int &ucap) {
            NL_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
            { k_max_seg<<<blocks_for(n, 256), 256, 0, s>>>(ptr, n, mx); nl_count_launch(); }
            NL_CHECK_LAUNCH();
            NL_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
            NL_CUDA(cudaStreamSynchronize(s));
            ucap = 32;
            while (ucap < (int64_t)hmx && ucap < UCAP) ucap <<= 1;
            hcap = std::min(HCAP, 2 * ucap);
        };
        int hcap1 = HCAP, ucap1 = UCAP;
        { k_elem_nodes<0><<<(unsigned)nt, GB, hsm0, s>>>(N, HCAP, UCAP, cnt, nullptr, nullptr, ovf); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        check_overflow();
        int64_t *nn_ptr = sc.get<int64_t>(nt + 1);
        int64_t nn_total = nl_scan_counts(cnt, nn_ptr, nt, &P->arena, s);
        int32_t *nn_ent = sc.get<int32_t>(nn_total);
        fill_shape(nn_ptr, nt, hcap1, ucap1);
        { k_elem_nodes<1><<<(unsigned)nt, GB, sizeof(int32_t) * (hcap1 + ucap1), s>>>(N, hcap1, ucap1, nullptr, nn_ptr,
                                                                                    nn_ent, ovf); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        { k_rows<0><<<(unsigned)nv, GB, hsm0, s>>>(N, HCAP, UCAP, m->ne_ptr, m->ne_ent, nn_ptr, nn_ent, cnt, nullptr,
                                                   nullptr, ovf); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        check_overflow();
        P->rowptr = P->arena.get<int64_t>(nv + 1);
        P->nnz = nl_scan_counts(cnt, P->rowptr, nv, &P->arena, s);
        NL_REQUIRE(P->nnz < 0x7fffffffLL, "nnz %lld exceeds the int32 position index", (long long)P->nnz);
        P->col = P->arena.get<int32_t>(P->nnz);
        fill_shape(P->rowptr, nv, hcap1, ucap1);
        { k_rows<1><<<(unsigned)nv, GB, sizeof(int32_t) * (hcap1 + ucap1), s>>>(N, hcap1, ucap1, m->ne_ptr, m->ne_ent,
                                                                            nn_ptr, nn_ent, nullptr, P->rowptr, P->col,
                                                                            ovf); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        check_overflow();

        NL_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
        { k_row_len_max<<<blocks_for(nv, 256), 256, 0, s>>>(P->rowptr, nv, mx); nl_count_launch(); }
        NL_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));

        P->perm = P->arena.get<int32_t>(P->nnz);
        int *bad = sc.get<int>(1);
        NL_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        { k_perm<<<(unsigned)nv, 128, 0, s>>>(P->rowptr, P->col, nv, P->perm, bad); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        P->elem_pos = P->arena.get<int32_t>(16 * nt);
        { k_elem_pos<<<blocks_for(nt, 128), 128, 0, s>>>(N, P->rowptr, P->col, P->elem_pos, bad); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        int64_t *slen = sc.get<int64_t>(4 * no);
        { k_strip_len<<<blocks_for(no, 128), 128, 0, s>>>(m->tets, m->outer_ids, P->rowptr, no, slen); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        P->strip_off = P->arena.get<int64_t>(4 * no + 1);
        P->strip_total = nl_scan_counts(slen, P->strip_off, 4 * no, &P->arena, s);

        // A = K[free, free]
        const int64_t nf = m->n_free;
        { k_a_count<false><<<blocks_for(nf, 128), 128, 0, s>>>(P->rowptr, P->col, m->free_nodes, m->free_idx, nf, cnt); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        P->a_rowptr = P->arena.get<int64_t>(nf + 1);
        P->nnz_a = nl_scan_counts(cnt, P->a_rowptr, nf, &P->arena, s);
        P->a_col = P->arena.get<int32_t>(P->nnz_a);
        P->a_src = P->arena.get<int32_t>(P->nnz_a);
        { k_a_fill<false><<<blocks_for(nf, 128), 128, 0, s>>>(P->rowptr, P->col, m->free_nodes, m->free_idx, nf, P->a_rowptr,
                                                       P->a_col, P->a_src); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        // A with its rows padded for the CG's vector loads
        int64_t *len4 = sc.get<int64_t>(std::max<int64_t>(nf, 1));
        { k_ap_len<<<blocks_for(nf, 256), 256, 0, s>>>(P->a_rowptr, nf, len4); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        P->ap_rowptr4 = P->arena.get<int64_t>(nf + 1);
        P->ap_slots = 4 * nl_scan_counts(len4, P->ap_rowptr4, nf, &P->arena, s);
        P->ap_col = P->arena.get<int32_t>(std::max<int64_t>(P->ap_slots, 4));
        P->ap_src = P->arena.get<int32_t>(std::max<int64_t>(P->ap_slots, 4));
        if (nf > 0) {
            { k_ap_fill<<<(unsigned)nf, 128, 0, s>>>(P->a_rowptr, P->a_col, nf, P->ap_rowptr4, P->ap_col, P->ap_src); nl_count_launch(); }
            NL_CHECK_LAUNCH();
        }
        // L = K[free, collar]: the lift of the volume constraint (b = F - L g)
        int64_t *lcnt = sc.get<int64_t>(std::max<int64_t>(nf, 1));
        { k_a_count<true><<<blocks_for(nf, 128), 128, 0, s>>>(P->rowptr, P->col, m->free_nodes, m->free_idx, nf, lcnt); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        P->l_rowptr = P->arena.get<int64_t>(nf + 1);
        P->nnz_l = nl_scan_counts(lcnt, P->l_rowptr, nf, &P->arena, s);
        P->l_col = P->arena.get<int32_t>(std::max<int64_t>(P->nnz_l, 1));
        P->l_src = P->arena.get<int32_t>(std::max<int64_t>(P->nnz_l, 1));
        { k_a_fill<true><<<blocks_for(nf, 128), 128, 0, s>>>(P->rowptr, P->col, m->free_nodes, m->free_idx, nf, P->l_rowptr,
                                                      P->l_col, P->l_src); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        int hbad = 0;
        NL_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        P->max_row = (int32_t)hmx;
        NL_REQUIRE(hbad == 0, "internal: sparsity pattern is not symmetric (%d)", hbad);
        NL_REQUIRE(P->max_row <= 65535, "a row of %d columns exceeds 65535", P->max_row);
    } catch (NlError &e) {
        P->arena.release_all();
        delete P;
        return e.st;
    }
    *out = P;
    return NL_OK;
}

extern "C" nl_status nl_pairs_build(nl_mesh *mesh, double delta, nl_pairs **out)
{
    nl_clear_error();
    if (!mesh || !out) { nl_set_error("NULL argument"); return NL_EINVAL; }
    *out = nullptr;
    if (!(delta > 0.0) || !isfinite(delta)) { nl_set_error("delta must be positive and finite"); return NL_EINVAL; }
    return nl_pairs_build_impl(mesh, delta, out);
}

extern "C" void nl_pairs_destroy(nl_pairs *p)
{
    if (!p) return;
    p->arena.release_all();
    delete p;
}

extern "C" nl_status nl_pairs_get_info(const nl_pairs *p, nl_pairs_info *info)
{
    nl_clear_error();
    if (!p || !info) { nl_set_error("NULL argument"); return NL_EINVAL; }
    info->n_vert = p->mesh->nv;
    info->n_tet = p->mesh->nt;
    info->n_outer = p->mesh->n_outer;
    info->n_pairs = p->npairs;
    info->nnz = p->nnz;
    info->n_free = p->mesh->n_free;
    info->nnz_a = p->nnz_a;
    info->nnz_lift = p->nnz_l;
    info->max_row = p->max_row;
    info->delta = p->delta;
    return NL_OK;
}

extern "C" nl_status nl_pairs_export(const nl_pairs *p, int32_t *outer, int64_t *ptr, int32_t *tp, int where)
{
    nl_clear_error();
    if (!p) { nl_set_error("NULL argument"); return NL_EINVAL; }
    if (where != NL_HOST && where != NL_DEVICE) { nl_set_error("bad where"); return NL_EINVAL; }
    cudaMemcpyKind kind = (where == NL_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaStream_t s = p->arena.stream();
    try {
        if (outer) NL_CUDA(cudaMemcpyAsync(outer, p->mesh->outer_ids, sizeof(int32_t) * p->mesh->n_outer, kind, s));
        if (ptr) NL_CUDA(cudaMemcpyAsync(ptr, p->pair_ptr, sizeof(int64_t) * (p->mesh->n_outer + 1), kind, s));
        if (tp) NL_CUDA(cudaMemcpyAsync(tp, p->pair_tp, sizeof(int32_t) * p->npairs, kind, s));
        NL_CUDA(cudaStreamSynchronize(s));
    } catch (NlError &e) {
        return e.st;
    }
    return NL_OK;
}
