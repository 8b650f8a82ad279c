// Assembly kernel: one thread block per outer element T (persistent loop),
// one thread per pair (T, T').  Per pair and outer point x_q the inner
// moments of the approximate ball inside T' are computed (nl_quad.cuh) and
// turned into the local block of Eq. (replaceBasis):
//   TT   += c * omega * lambda(x_q) lambda(x_q)^T m0      (summed per T)
//   TT'  -= c * omega * lambda(x_q) m1^T                   (cross strip of T)
//   T'T' += c * omega * m2                                  (staged per pair)
// with c = (gamma/2) |T|/4 and omega = 2 for collar elements T'.
//
// Determinism: the cross contributions of a chunk of pairs are added into
// the strips (the four CSR rows of T's nodes, in shared memory) by one warp
// per row in pair order; everything else is written to its own slot.
#pragma once

#include "nl_internal.h"
#include "nl_quad.cuh"

namespace nla {

using nlq::Mom;
using nlq::P3;

struct AsmArgs {
    const double4 *verts;
    const float4 *vhi, *vlo;
    const int4 *tets;
    const uint8_t *in_omega;
    const double *tet_vol;
    const int32_t *outer_ids;
    const double *xq;
    const int64_t *pair_ptr;
    const int32_t *pair_tp;
    const int64_t *rowptr;
    const int32_t *col;
    const int64_t *strip_off;
    int64_t n_outer;
    int max_row;
    double delta2;
    double half_gamma;
    int nmc;
    uint2 key;
    void *D;                 // [npairs][10] staged T'T' moments (R)
    double *strips;          // [strip_total]
    double *TT;              // [n_outer][10]
    unsigned long long *stats;  // [5]
};

constexpr int NT = 128;      // threads per block = pairs per chunk

__device__ __forceinline__ int lower_bound_s(const int32_t *a, int n, int32_t key)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// barycentric weight lambda_i(x_q) of the 4-point rule: a on i == q, b elsewhere
template <class R> __device__ __forceinline__ R qlam(int i, int q)
{
    return (i == q) ? R(0x1.2bbae2a27f931p-1) : R(0x1.1b06d1d200913p-3);
}

template <class R, int STRAT>
__global__ void __launch_bounds__(NT) k_assemble(AsmArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int mr = A.max_row;
    int32_t *cols = reinterpret_cast<int32_t *>(smem);                       // [4][mr]
    double *strip = reinterpret_cast<double *>(smem + sizeof(int32_t) * 4 * ((mr + 1) & ~1));  // [4][mr]
    R *Xs = reinterpret_cast<R *>(strip + 4 * mr);                            // [NT][16]
    int32_t *offs = reinterpret_cast<int32_t *>(Xs + NT * 16);                // [NT][16]
    double *wsc = reinterpret_cast<double *>(offs + NT * 16);                 // [NT]
    double *red = wsc + NT;                                                   // [NT/32][4]
    __shared__ int lens[4];
    __shared__ unsigned long long sstat[5];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    nlq::Stats st{0, 0, 0, 0, 0};

    for (int64_t o = blockIdx.x; o < A.n_outer; o += gridDim.x) {
        const int32_t T = A.outer_ids[o];
        const int4 eT = A.tets[T];
        const int nodeT[4] = {eT.x, eT.y, eT.z, eT.w};
        if (tid < 4) lens[tid] = (int)(A.rowptr[nodeT[tid] + 1] - A.rowptr[nodeT[tid]]);
        __syncthreads();
        for (int i = 0; i < 4; ++i) {
            const int64_t rb = A.rowptr[nodeT[i]];
            for (int c = tid; c < lens[i]; c += NT) {
                cols[i * mr + c] = A.col[rb + c];
                strip[i * mr + c] = 0.0;
            }
        }
        double xqd[4][3];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int d = 0; d < 3; ++d) xqd[q][d] = A.xq[12 * o + 3 * q + d];
        const double cT = A.half_gamma * (A.tet_vol[T] * 0.25);
        double vq[4] = {0.0, 0.0, 0.0, 0.0};
        __syncthreads();

        const int64_t pb = A.pair_ptr[o], pe = A.pair_ptr[o + 1];
        for (int64_t base = pb; base < pe; base += NT) {
            const int cnt = (int)((pe - base) < (int64_t)NT ? (pe - base) : (int64_t)NT);
            const int64_t p = base + tid;
            if (tid < cnt) {
                const int32_t Tp = A.pair_tp[p];
                const int4 eP = A.tets[Tp];
                const int nodeP[4] = {eP.x, eP.y, eP.z, eP.w};
                const double omega = A.in_omega[Tp] ? 1.0 : 2.0;
                const R volTp = (R)A.tet_vol[Tp];
                R Y[4][4], V[4], Dp[10];
#pragma unroll
                for (int k = 0; k < 10; ++k) Dp[k] = R(0);
                P3<R> v[4];
                if (sizeof(R) == 8) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        double4 g = A.verts[nodeP[k]];
                        v[k] = nlq::mk3<R>((R)g.x, (R)g.y, (R)g.z);
                    }
                }
                float4 vh[4], vl[4];
                if (sizeof(R) == 4) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) { vh[k] = A.vhi[nodeP[k]]; vl[k] = A.vlo[nodeP[k]]; }
                }
#pragma unroll 1
                for (int q = 0; q < 4; ++q) {
                    P3<R> x;
                    P3<R> vv[4];
                    if (sizeof(R) == 8) {
                        x = nlq::mk3<R>((R)xqd[q][0], (R)xqd[q][1], (R)xqd[q][2]);
#pragma unroll
                        for (int k = 0; k < 4; ++k) vv[k] = v[k];
                    } else {
                        // coordinates relative to x_q as double-float differences
                        float xh[3], xl[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            xh[d] = (float)xqd[q][d];
                            xl[d] = (float)(xqd[q][d] - (double)xh[d]);
                        }
                        x = nlq::mk3<R>(R(0), R(0), R(0));
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            vv[k] = nlq::mk3<R>((R)((vh[k].x - xh[0]) + (vl[k].x - xl[0])),
                                                (R)((vh[k].y - xh[1]) + (vl[k].y - xl[1])),
                                                (R)((vh[k].z - xh[2]) + (vl[k].z - xl[2])));
                    }
                    Mom<R> M;
                    nlq::Strict sx;
                    if (sizeof(R) == 4) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            double4 g = A.verts[nodeP[k]];
                            sx.v[k][0] = g.x; sx.v[k][1] = g.y; sx.v[k][2] = g.z;
                        }
                        sx.x[0] = xqd[q][0]; sx.x[1] = xqd[q][1]; sx.x[2] = xqd[q][2];
                        sx.d2 = A.delta2;
                    }
                    nlq::point_moments<R, STRAT>(vv, x, (R)A.delta2, volTp, A.nmc, A.key, (uint32_t)T, (uint32_t)Tp,
                                                 (uint32_t)q, M, st, sizeof(R) == 4 ? &sx : nullptr);
                    V[q] = M.m0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) Y[q][k] = M.m1[k];
#pragma unroll
                    for (int k = 0; k < 10; ++k) Dp[k] += M.m2[k];
                }
                // staged T'T' moments (scaled later by c * omega)
                R *Dst = reinterpret_cast<R *>(A.D) + 10 * p;
#pragma unroll
                for (int k = 0; k < 10; ++k) Dst[k] = Dp[k];
#pragma unroll
                for (int q = 0; q < 4; ++q) vq[q] += omega * (double)V[q];
                // cross: X[i][k] = sum_q lambda_i(x_q) m1_k(q)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        R s = ((qlam<R>(i, 0) * Y[0][k] + qlam<R>(i, 1) * Y[1][k]) + qlam<R>(i, 2) * Y[2][k]) +
                              qlam<R>(i, 3) * Y[3][k];
                        Xs[tid * 16 + 4 * i + k] = s;
                    }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) offs[tid * 16 + 4 * i + k] = lower_bound_s(cols + i * mr, lens[i], nodeP[k]);
                wsc[tid] = -(omega * cT);
            }
            __syncthreads();
            // deterministic strip accumulation: warp i owns row i; pairs in order
            {
                const int i = warp;
                for (int t = 0; t < cnt; ++t) {
                    if (lane < 4) {
                        const int c = offs[t * 16 + 4 * i + lane];
                        strip[i * mr + c] += wsc[t] * (double)Xs[t * 16 + 4 * i + lane];
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
        }
        // TT block: c * sum_q lambda(x_q) lambda(x_q)^T V_q, with V_q summed over the block in fixed order
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double s = vq[q];
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) red[warp * 4 + q] = s;
        }
        __syncthreads();
        if (tid < 10) {
            double V[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) V[q] = (red[0 * 4 + q] + red[1 * 4 + q]) + (red[2 * 4 + q] + red[3 * 4 + q]);
            const int ia[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
            const int ib[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
            const int i = ia[tid], j = ib[tid];
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q) s += qlam<double>(i, q) * qlam<double>(j, q) * V[q];
            A.TT[10 * o + tid] = cT * s;
        }
        // strips out
        for (int i = 0; i < 4; ++i) {
            const int64_t so = A.strip_off[4 * o + i];
            for (int c = tid; c < lens[i]; c += NT) A.strips[so + c] = strip[i * mr + c];
        }
        __syncthreads();
    }
    // statistics (integer atomics)
    if (tid < 5) sstat[tid] = 0ULL;
    __syncthreads();
    atomicAdd(&sstat[0], (unsigned long long)st.cut);
    atomicAdd(&sstat[1], (unsigned long long)st.inside);
    atomicAdd(&sstat[2], (unsigned long long)st.mc);
    atomicAdd(&sstat[3], (unsigned long long)st.acc);
    atomicAdd(&sstat[4], (unsigned long long)st.fallback);
    __syncthreads();
    if (tid < 5 && sstat[tid]) atomicAdd(&A.stats[tid], sstat[tid]);
}

inline size_t asm_smem_bytes(int max_row, size_t real_size)
{
    size_t b = sizeof(int32_t) * 4 * (size_t)((max_row + 1) & ~1);
    b += sizeof(double) * 4 * (size_t)max_row;
    b += real_size * NT * 16;
    b += sizeof(int32_t) * NT * 16;
    b += sizeof(double) * NT;
    b += sizeof(double) * (NT / 32) * 4;
    return b;
}

template <class R>
void launch_assemble(nl_system *sys, void *D, double *strips, double *TT, unsigned long long *stats)
{
    nl_pairs *P = sys->pairs;
    nl_mesh *m = P->mesh;
    AsmArgs A;
    A.verts = m->verts; A.vhi = m->vhi; A.vlo = m->vlo; A.tets = m->tets; A.in_omega = m->in_omega;
    A.tet_vol = m->tet_vol; A.outer_ids = m->outer_ids; A.xq = m->xq; A.pair_ptr = P->pair_ptr;
    A.pair_tp = P->pair_tp; A.rowptr = P->rowptr; A.col = P->col; A.strip_off = P->strip_off;
    A.n_outer = m->n_outer; A.max_row = P->max_row;
    A.delta2 = P->delta * P->delta;
    A.half_gamma = sys->opts.gamma / 2.0;
    A.nmc = sys->opts.strategy == NL_FULLCAPS ? sys->opts.mc_points : 0;
    A.key = make_uint2((uint32_t)sys->opts.seed, (uint32_t)(sys->opts.seed >> 32));
    A.D = D; A.strips = strips; A.TT = TT; A.stats = stats;
    size_t smem = asm_smem_bytes(P->max_row, sizeof(R));
    NL_REQUIRE(smem <= 220 * 1024, "rows of %d columns need %zu bytes of shared memory", P->max_row, smem);
    void (*kern)(AsmArgs) = nullptr;
    switch (sys->opts.strategy) {
    case NL_NOCAPS: kern = k_assemble<R, 0>; break;
    case NL_APPROXCAPS: kern = k_assemble<R, 1>; break;
    default: kern = k_assemble<R, 2>; break;
    }
    NL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    per_sm = per_sm < 1 ? 1 : per_sm;
    int64_t grid = (int64_t)nl_num_sms() * per_sm;
    if (grid > m->n_outer) grid = m->n_outer;
    { kern<<<(unsigned)grid, NT, smem, sys->arena.stream()>>>(A); nl_count_launch(); }
    NL_CHECK_LAUNCH();
}

}  // namespace nla

namespace nla {

// Diagnostic kernel: moments of one (T', x) case per thread, with the same
// device code (and, per translation unit, the same compiler flags) as the
// assembly kernel.  For float, coordinates are made relative to x as
// double-float differences exactly as in the assembly.
template <class R, int STRAT>
__global__ void k_probe(const double *__restrict__ tv, const double *__restrict__ xs, const uint32_t *__restrict__ ids,
                        int64_t n, double delta2, int nmc, uint2 key, double *out)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double *t = tv + 12 * c;
    double x[3] = {xs[3 * c], xs[3 * c + 1], xs[3 * c + 2]};
    P3<R> v[4];
    P3<R> xx;
    nlq::P3<double> vd[4];
    for (int k = 0; k < 4; ++k) vd[k] = nlq::mk3<double>(t[3 * k], t[3 * k + 1], t[3 * k + 2]);
    double vol = nlq::vol4(vd[0], vd[1], vd[2], vd[3]);
    if (sizeof(R) == 8) {
        for (int k = 0; k < 4; ++k) v[k] = nlq::mk3<R>((R)vd[k].x, (R)vd[k].y, (R)vd[k].z);
        xx = nlq::mk3<R>((R)x[0], (R)x[1], (R)x[2]);
    } else {
        float xh[3], xl[3];
        for (int d = 0; d < 3; ++d) { xh[d] = (float)x[d]; xl[d] = (float)(x[d] - (double)xh[d]); }
        for (int k = 0; k < 4; ++k) {
            double g[3] = {vd[k].x, vd[k].y, vd[k].z};
            float h[3], l[3];
            for (int d = 0; d < 3; ++d) { h[d] = (float)g[d]; l[d] = (float)(g[d] - (double)h[d]); }
            v[k] = nlq::mk3<R>((R)((h[0] - xh[0]) + (l[0] - xl[0])), (R)((h[1] - xh[1]) + (l[1] - xl[1])),
                               (R)((h[2] - xh[2]) + (l[2] - xl[2])));
        }
        xx = nlq::mk3<R>(R(0), R(0), R(0));
    }
    Mom<R> M;
    nlq::Stats st{0, 0, 0, 0, 0};
    nlq::Strict sx;
    for (int k = 0; k < 4; ++k) { sx.v[k][0] = vd[k].x; sx.v[k][1] = vd[k].y; sx.v[k][2] = vd[k].z; }
    for (int d = 0; d < 3; ++d) sx.x[d] = x[d];
    sx.d2 = delta2;
    nlq::point_moments<R, STRAT>(v, xx, (R)delta2, (R)vol, nmc, key, ids[3 * c], ids[3 * c + 1], ids[3 * c + 2], M, st,
                                 sizeof(R) == 4 ? &sx : nullptr);
    out[15 * c] = (double)M.m0;
    for (int k = 0; k < 4; ++k) out[15 * c + 1 + k] = (double)M.m1[k];
    for (int k = 0; k < 10; ++k) out[15 * c + 5 + k] = (double)M.m2[k];
}

template <class R>
void launch_probe(const double *tv, const double *xs, const uint32_t *ids, int64_t n, double delta2, int strategy,
                  int nmc, uint64_t seed, double *out)
{
    uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    unsigned blocks = (unsigned)((n + 127) / 128);
    if (strategy == NL_NOCAPS) { k_probe<R, 0><<<blocks, 128>>>(tv, xs, ids, n, delta2, 0, key, out); nl_count_launch(); }
    else if (strategy == NL_APPROXCAPS) { k_probe<R, 1><<<blocks, 128>>>(tv, xs, ids, n, delta2, 0, key, out); nl_count_launch(); }
    else { k_probe<R, 2><<<blocks, 128>>>(tv, xs, ids, n, delta2, nmc, key, out); nl_count_launch(); }
    NL_CHECK_LAUNCH();
}

}  // namespace nla
