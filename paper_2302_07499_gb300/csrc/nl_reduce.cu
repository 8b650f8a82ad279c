// Deterministic reduction of the assembly outputs into the CSR matrix K,
// the free block A = K[free,free] and the right-hand side b (no floating-
// point atomics: every sum runs in a fixed order).
//
//   G  = sum over outer elements of their cross strips (row gather)
//   K  = G + G^T + sum over elements of their 4x4 element blocks
//        (TT of the outer element plus the T'T' moments of every pair that
//        has the element as T', scaled by omega (gamma/2)|T|/4)
//   F_i = sum_T sum_q (|T|/4) lambda_i(x_q) f            (Alg. 5, last save)
//   b  = F[free] - K[free, collar] g[collar]
#include <algorithm>

#include "nl_internal.h"
#include "nl_df.cuh"

namespace {

// G row r = sum over outer elements T containing r (increasing id) of the
// strip of T for r's local index.  One warp per row, lanes over columns.
__global__ void k_strip_gather(const int64_t *__restrict__ rowptr, const int64_t *__restrict__ ne_ptr,
                               const int32_t *__restrict__ ne_ent, const int32_t *__restrict__ outer_of,
                               const int64_t *__restrict__ strip_off, const double *__restrict__ strips, int64_t nv,
                               double *G)
{
    int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (r >= nv) return;
    int64_t rb = rowptr[r];
    int len = (int)(rowptr[r + 1] - rb);
    for (int c0 = 0; c0 < len; c0 += 32 * 4) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t k = ne_ptr[r]; k < ne_ptr[r + 1]; ++k) {
            int32_t ent = ne_ent[k];
            int32_t o = outer_of[ent >> 2];
            if (o < 0) continue;
            const double *s = strips + strip_off[4 * (int64_t)o + (ent & 3)];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int c = c0 + u * 32 + lane;
                if (c < len) acc[u] += s[c];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int c = c0 + u * 32 + lane;
            if (c < len) G[rb + c] = acc[u];
        }
    }
}

// element blocks: warp per element; lanes take pairs lane, lane+32, ...;
// fixed butterfly reduction.  Layout of the 10 values: (0,0) (0,1) (0,2)
// (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3).  FP64 path: D holds each pair's
// full T'T' moments.
__global__ void k_elem_blocks(const int64_t *__restrict__ tp_ptr, const int32_t *__restrict__ tp_pair,
                              const int32_t *__restrict__ pair_T, const double *__restrict__ tet_vol,
                              const uint8_t *__restrict__ in_omega, const int32_t *__restrict__ outer_of,
                              const double *__restrict__ D, const double *__restrict__ TT, double half_gamma, int64_t nt,
                              double *E)
{
    int64_t el = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (el >= nt) return;
    double omega = in_omega[el] ? 1.0 : 2.0;
    double acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.0;
    for (int64_t j = tp_ptr[el] + lane; j < tp_ptr[el + 1]; j += 32) {
        int32_t p = tp_pair[j];
        double w = omega * (half_gamma * (tet_vol[pair_T[p]] * 0.25));
        const double *d = D + 10 * (int64_t)p;
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] += w * d[k];
    }
#pragma unroll
    for (int k = 0; k < 10; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    if (lane < 10) {
        double v = acc[0];
#pragma unroll
        for (int k = 1; k < 10; ++k)
            if (lane == k) v = acc[k];
        int32_t o = outer_of[el];
        if (o >= 0) v += TT[10 * (int64_t)o + lane];
        E[10 * el + lane] = v;
    }
}

// The same for the FP32 path, with double-float sums (FP32 pipes only): the
// weight w = omega (gamma/2) |T| / 4 from |T| as float hi + lo, the 10
// staged FP32 values of each pair, and the points at which T' = el is whole
// (nfull per pair, kept out of the FP32 staging) as the sum of their weights
// scaled once by |T'|(1 + delta_ab)/20.
__global__ void k_elem_blocks_df(const int64_t *__restrict__ tp_ptr, const int32_t *__restrict__ tp_pair,
                                 const int32_t *__restrict__ pair_T, const double *__restrict__ tet_vol,
                                 const float2 *__restrict__ vol_hl, const uint8_t *__restrict__ in_omega,
                                 const int32_t *__restrict__ outer_of, const float *__restrict__ D,
                                 const uint8_t *__restrict__ nfull, const double *__restrict__ Dw,
                                 const double *__restrict__ TT, double half_gamma, int64_t nt, double *E)
{
    using nla::DF;
    int64_t el = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (el >= nt) return;
    const float omega = in_omega[el] ? 1.f : 2.f;
    const DF hg4 = nla::df_from(half_gamma * 0.25);
    DF acc[10], sw{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = DF{0.f, 0.f};
    for (int64_t j = tp_ptr[el] + lane; j < tp_ptr[el + 1]; j += 32) {
        const int32_t p = tp_pair[j];
        const float2 vh = vol_hl[pair_T[p]];
        const DF w = nla::df_mul(nla::df_mul2(hg4, DF{vh.x, vh.y}), omega);
        const float *d = D + 10 * (int64_t)p;
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] = nla::df_add(acc[k], nla::df_mul(w, d[k]));
        if (nfull) sw = nla::df_add(sw, nla::df_mul(w, (float)nfull[p]));
        if (Dw) {
            // kernel shapes: the whole-T' points' moments, in FP64
            const double *dw = Dw + 10 * (int64_t)p;
#pragma unroll
            for (int k = 0; k < 10; ++k) acc[k] = nla::df_add(acc[k], nla::df_mul2(w, nla::df_from(dw[k])));
        }
    }
#pragma unroll
    for (int k = 0; k < 10; ++k)
        for (int off = 16; off > 0; off >>= 1)
            acc[k] = nla::df_add(acc[k], DF{__shfl_xor_sync(0xffffffffu, acc[k].hi, off),
                                            __shfl_xor_sync(0xffffffffu, acc[k].lo, off)});
    for (int off = 16; off > 0; off >>= 1)
        sw = nla::df_add(sw, DF{__shfl_xor_sync(0xffffffffu, sw.hi, off), __shfl_xor_sync(0xffffffffu, sw.lo, off)});
    if (lane < 10) {
        DF a = acc[0];
#pragma unroll
        for (int k = 1; k < 10; ++k)
            if (lane == k) a = acc[k];
        const double cf = (lane == 0 || lane == 4 || lane == 7 || lane == 9) ? 0.1 : 0.05;
        double v = nla::df_to(a) + nla::df_to(sw) * (tet_vol[el] * cf);
        int32_t o = outer_of[el];
        if (o >= 0) v += TT[10 * (int64_t)o + lane];
        E[10 * el + lane] = v;
    }
}

__device__ __forceinline__ int sym10(int i, int j)
{
    int a = i < j ? i : j, b = i < j ? j : i;
    // offsets of row a in the upper triangle: 0, 4, 7, 9
    int base = (a == 0) ? 0 : (a == 1) ? 4 : (a == 2) ? 7 : 9;
    return base + (b - a);
}

// K row r = G + G^T over the row, then the element blocks of the active
// elements around r in increasing element id.
__global__ void k_final_K(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ perm,
                          const double *__restrict__ G, const int64_t *__restrict__ ne_ptr,
                          const int32_t *__restrict__ ne_ent, const int32_t *__restrict__ elem_pos,
                          const double *__restrict__ E, int64_t nv, double *K)
{
    int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (r >= nv) return;
    for (int64_t e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32) K[e] = G[e] + G[perm[e]];
    __syncwarp();
    for (int64_t k = ne_ptr[r]; k < ne_ptr[r + 1]; ++k) {
        int32_t ent = ne_ent[k];
        int64_t el = ent >> 2;
        int i = ent & 3;
        if (lane < 4) {
            int32_t pos = elem_pos[16 * el + 4 * i + lane];
            if (pos >= 0) K[pos] += E[10 * el + sym10(i, lane)];
        }
        __syncwarp();
    }
}

// F_r = sum over elements T of Omega holding node r of sum_q w_q lambda_r(x_q)
// f(x_q), with f = fconst + the P1 interpolant of the nodal values fnod
// (when given) and lambda(x_q) = a at point q, b at the other three.
__global__ void k_load_vector(const int64_t *__restrict__ ne_ptr, const int32_t *__restrict__ ne_ent,
                              const int32_t *__restrict__ outer_of, const double *__restrict__ tet_vol,
                              const int4 *__restrict__ tets, const double *__restrict__ fnod, double fconst,
                              int64_t nv, double *F)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nv) return;
    const double qa = 0x1.2bbae2a27f931p-1, qb = 0x1.1b06d1d200913p-3;
    double s = 0.0;
    for (int64_t k = ne_ptr[r]; k < ne_ptr[r + 1]; ++k) {
        int32_t ent = ne_ent[k];
        int64_t el = ent >> 2;
        if (outer_of[el] < 0) continue;
        const int i = ent & 3;
        double w = tet_vol[el] * 0.25;
        double fq[4] = {fconst, fconst, fconst, fconst};
        if (fnod) {
            const int4 t = tets[el];
            const double f4[4] = {fnod[t.x], fnod[t.y], fnod[t.z], fnod[t.w]};
            for (int q = 0; q < 4; ++q) {
                double v = 0.0;
                for (int j = 0; j < 4; ++j) v += (j == q ? qa : qb) * f4[j];
                fq[q] += v;
            }
        }
        // sum over the four points: lambda_i = a at its own point, b at the others
        double t = 0.0;
        for (int q = 0; q < 4; ++q) t += w * (q == i ? qa : qb) * fq[q];
        s += t;
    }
    F[r] = s;
}

__global__ void k_system(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                         const double *__restrict__ K, const int32_t *__restrict__ free_nodes,
                         const int32_t *__restrict__ free_idx, const int64_t *__restrict__ a_rowptr,
                         const int32_t *__restrict__ a_src, const double *__restrict__ F,
                         const double *__restrict__ g, int64_t n_free, double *Aval, float *A32, double *b)
{
    int64_t fr = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (fr >= n_free) return;
    for (int64_t e = a_rowptr[fr] + lane; e < a_rowptr[fr + 1]; e += 32) {
        double v = K[a_src[e]];
        Aval[e] = v;
        A32[e] = (float)v;
    }
    int32_t r = free_nodes[fr];
    double s = 0.0;
    for (int64_t e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32) {
        int32_t c = col[e];
        if (free_idx[c] < 0) s += K[e] * g[c];
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) b[fr] = F[r] - s;
}

// A's values in the padded rows (0 for the pads), FP64 and FP32
__global__ void k_fill_padded(const double *__restrict__ A, const int32_t *__restrict__ src, int64_t n, double *Ap,
                              float *Ap32)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int32_t k = src[e];
    const double v = k >= 0 ? A[k] : 0.0;
    Ap[e] = v;
    Ap32[e] = (float)v;
}

// out[e] = K[src[e]] (a row view's values)
__global__ void k_gather_vals(const double *__restrict__ K, const int32_t *__restrict__ src, int64_t n, double *out)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = K[src[e]];
}

unsigned wblocks(int64_t n) { return (unsigned)std::max<int64_t>(1, nl_cdiv<int64_t>(n * 32, 256)); }

}  // namespace

// The reduction into K, A, b with caller-given scratch G [nnz] and E [10 nt]
// (stream-ordered, no synchronisation: capturable in a CUDA graph).
void nl_reduce_system_into(nl_system *sys, const void *D, int d_is_float, const uint8_t *nfull, const double *strips,
                           const double *TT, double *G, double *E, cudaStream_t s)
{
    nl_pairs *P = sys->pairs;
    nl_mesh *m = P->mesh;
    { k_strip_gather<<<wblocks(m->nv), 256, 0, s>>>(P->rowptr, m->ne_ptr, m->ne_ent, m->outer_of, P->strip_off, strips,
                                                 m->nv, G); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    if (d_is_float)
        { k_elem_blocks_df<<<wblocks(m->nt), 256, 0, s>>>(P->tp_ptr, P->tp_pair, P->pair_T, m->tet_vol, m->vol_hl,
                                                         m->in_omega, m->outer_of, (const float *)D, nfull, sys->Dw,
                                                         TT, sys->opts.gamma / 2.0, m->nt, E); nl_count_launch(); }
    else
        { k_elem_blocks<<<wblocks(m->nt), 256, 0, s>>>(P->tp_ptr, P->tp_pair, P->pair_T, m->tet_vol, m->in_omega,
                                                    m->outer_of, (const double *)D, TT, sys->opts.gamma / 2.0, m->nt,
                                                    E); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    { k_final_K<<<wblocks(m->nv), 256, 0, s>>>(P->rowptr, P->perm, G, m->ne_ptr, m->ne_ent, P->elem_pos, E, m->nv,
                                            sys->K); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    { k_load_vector<<<(unsigned)nl_cdiv<int64_t>(m->nv, 256), 256, 0, s>>>(m->ne_ptr, m->ne_ent, m->outer_of,
                                                                       m->tet_vol, m->tets, sys->f, sys->opts.f_const,
                                                                       m->nv, sys->F); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    { k_system<<<wblocks(m->n_free), 256, 0, s>>>(P->rowptr, P->col, sys->K, m->free_nodes, m->free_idx, P->a_rowptr,
                                               P->a_src, sys->F, sys->g, m->n_free, sys->A, sys->A32, sys->b); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    if (P->ap_slots > 0) {
        { k_fill_padded<<<(unsigned)nl_cdiv<int64_t>(P->ap_slots, 256), 256, 0, s>>>(sys->A, P->ap_src, P->ap_slots,
                                                                                  sys->Ap, sys->Ap32); nl_count_launch(); }
        NL_CHECK_LAUNCH();
    }
    if (P->nnz_l > 0) {
        { k_gather_vals<<<(unsigned)nl_cdiv<int64_t>(P->nnz_l, 256), 256, 0, s>>>(sys->K, P->l_src, P->nnz_l, sys->L); nl_count_launch(); }
        NL_CHECK_LAUNCH();
    }
}

void nl_reduce_system(nl_system *sys, const void *D, int d_is_float, const uint8_t *nfull, const double *strips,
                      const double *TT)
{
    nl_pairs *P = sys->pairs;
    nl_mesh *m = P->mesh;
    Scratch sc(&sys->arena);
    double *G = sc.get<double>(P->nnz);
    double *E = sc.get<double>(10 * m->nt);
    nl_reduce_system_into(sys, D, d_is_float, nfull, strips, TT, G, E, sys->arena.stream());
    // scratch is released (stream-ordered) when sc goes out of scope
    NL_CUDA(cudaStreamSynchronize(sys->arena.stream()));
}
