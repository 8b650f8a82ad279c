// Quadrature of the nonlocal assembly, three kernels per chunk of
// (pair, point) units:
//   K1 k_classify  one thread per unit (pair, outer point x_q): classifies
//                  the vertices of T' against the ball around x_q and lists
//                  the units with a cut (1..3 vertices inside, or a fullcaps
//                  cap without inside vertices) per class;
//   K2 k_events    one thread per listed unit, warps of one class: the inner
//                  moments of the approximate ball inside T' (nl_quad.cuh);
//   K3 k_combine   one block per outer element T: the local block of
//                  Eq. (replaceBasis) from the moments of its pairs,
//     TT   += c * omega * lambda(x_q) lambda(x_q)^T m0      (summed per T)
//     TT'  -= c * omega * lambda(x_q) m1^T                   (cross strip of T)
//     T'T' += c * omega * m2                                  (staged per pair)
//   with c = (gamma/2) |T|/4 and omega = 2 for collar elements T'.
//
// Determinism: the cross contributions are added into the strips (the four
// CSR rows of T's nodes, in shared memory) in an order fixed by the pair
// order alone; everything else is written to its own slot.  A launch serves
// one problem or, through the pair -> problem map, a group of problems of a
// batch, with the same arithmetic per unit.
#pragma once

#include "nl_asm_types.h"
#include "nl_internal.h"
#include "nl_quad.cuh"
#include "nl_df.cuh"

#include <string.h>

#include <algorithm>
#include <vector>

namespace nla {

using nlq::Mom;
using nlq::P3;

// The problem of pair pg (launch index space) and the pair's own index in it.
template <bool B>
__device__ __forceinline__ const Prob &prob_of_pair(const AsmArgs &A, int64_t pg, int64_t &p)
{
    if constexpr (B) {
        const Prob &P = A.probs[A.pair_prob[pg]];
        p = pg - P.pair_base;
        return P;
    } else {
        p = pg;
        return A.self;
    }
}

// The problem of outer element og (launch index space) and its own index.
template <bool B>
__device__ __forceinline__ const Prob &prob_of_outer(const AsmArgs &A, int64_t og, int64_t &o)
{
    if constexpr (B) {
        const Prob &P = A.probs[A.outer_prob[og]];
        o = og - P.outer_base;
        return P;
    } else {
        o = og;
        return A.self;
    }
}

// barycentric weight lambda_i(x_q) of the 4-point rule: a on i == q, b elsewhere
template <class R> __device__ __forceinline__ R qlam(int i, int q)
{
    return (i == q) ? R(0x1.2bbae2a27f931p-1) : R(0x1.1b06d1d200913p-3);
}

// T' vertex coordinates for the point x_q: global FP64 (R = double) or
// relative to x_q as double-float differences (R = float), plus the FP64
// context for the FP32 path's exact decisions.
template <class R>
__device__ __forceinline__ void load_point_geometry(const Prob &A, int4 eP, int64_t o, int q, P3<R> v[4],
                                                    P3<R> &x, nlq::Strict &sx)
{
    const int ids[4] = {eP.x, eP.y, eP.z, eP.w};
    const double *xq = A.xq + 12 * o + 3 * q;
    if (sizeof(R) == 8) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double4 g = A.verts[ids[k]];
            v[k] = nlq::mk3<R>((R)g.x, (R)g.y, (R)g.z);
        }
        x = nlq::mk3<R>((R)xq[0], (R)xq[1], (R)xq[2]);
    } else {
        const float *xh = A.xq_hl + 24 * o + 6 * q;   // hi xyz, lo xyz
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 h = A.vhi[ids[k]], l = A.vlo[ids[k]];
            v[k] = nlq::mk3<R>((R)((h.x - xh[0]) + (l.x - xh[3])), (R)((h.y - xh[1]) + (l.y - xh[4])),
                               (R)((h.z - xh[2]) + (l.z - xh[5])));
        }
        x = nlq::mk3<R>(R(0), R(0), R(0));
        sx.verts = A.verts;
        sx.e = eP;
        sx.x = xq;
        sx.d2 = A.delta2;
    }
}

// ---------------------------------------------------------------------------
// K1: classify every (pair, point) unit of the chunk; units with a cut (1..3
// vertices inside, or a fullcaps cap without inside vertices) become events.
template <class R, int STRAT, bool B>
__global__ void __launch_bounds__(256, 3) k_classify(const __grid_constant__ AsmArgs A)
{
    const int64_t nu = 4 * (A.p1 - A.p0);
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nu; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = base + threadIdx.x;
        bool ev = false;
        uint8_t info = 0x20;
        if (u < nu) {
            int64_t p;
            const Prob &P = prob_of_pair<B>(A, A.p0 + (u >> 2), p);
            const int q = (int)(u & 3);
            const int32_t T = P.pair_T[p], Tp = P.pair_tp[p];
            const int32_t o = P.outer_of[T];
            P3<R> v[4];
            P3<R> x;
            nlq::Strict sx;
            load_point_geometry<R>(P, P.tets[Tp], o, q, v, x, sx);
            const nlq::Strict *sp = (sizeof(R) == 4) ? &sx : nullptr;
            const R d2 = (sizeof(R) == 4) ? (R)P.delta2f : (R)P.delta2;
            const int inm = nlq::classify(v, x, d2, sp);
            info = (uint8_t)inm;
            if constexpr (STRAT >= 3) {
                // element-level strategies: T' whole (closed form) or nothing
                info = nlq::element_full<R, STRAT>(v, x, d2, inm, sp) ? (uint8_t)15 : (uint8_t)0x20;
            } else if (inm != 15) {
                if (inm != 0) ev = true;
                else if (STRAT == 2 && A.nmc > 0) ev = nlq::meets_ball(v, x, d2, sp);
                if (ev) info |= 0x10;
                else info |= 0x20;
            }
            // kernel shapes: a whole T' gets a record too (k_whole_shape)
            if (A.kpoly && (info & 15) == 15) info = 15 | 0x10;
        }
        // warp-aggregated slot allocation within the event's class (number of
        // inside vertices), so that each warp of K2 runs one geometry case:
        // the lanes of one class find each other, their first lane reserves
        // the class's slots
        const int cls = __popc((unsigned)(info & 15));
        const unsigned grp = __match_any_sync(0xffffffffu, ev ? cls : -1);
        const int leader = __ffs(grp) - 1;
        int basep = 0;
        if (ev && lane == leader) basep = atomicAdd(&A.nev[cls], __popc(grp));
        basep = __shfl_sync(0xffffffffu, basep, leader);
        if (ev) {
            const int idx = basep + __popc(grp & ((1u << lane) - 1u));
            A.evu[cls * nu + idx] = (int32_t)u;
        }
        if (u < nu) A.uinfo[u] = info;
    }
}

// ---------------------------------------------------------------------------
// K2: one thread per event: cells of hull(I u P) and, for fullcaps, the
// Monte Carlo loop over the cap (uniform trip count across the warp).
template <class R> struct EvCfg {
    static constexpr int threads = sizeof(R) == 4 ? 128 : 64;
    // the cap cells, then a 17-value record stage per thread (odd stride:
    // conflict-free scalar accesses)
    static constexpr size_t smem = sizeof(R) * threads * (3 * nlq::CB_STRIDE + 17);
    // 4 resident blocks per SM: 128 registers a thread, no spills (the cap
    // scratch would allow 5 blocks at 96 registers; the spills that forces
    // cost more than the fifth block gains: 21.1 -> 19.5 ms on the bench step)
    static constexpr int min_blocks = 4;
};

// FP32 nocaps and fullcaps: events whose m = 2 diagonal needs the FP64
// retake are handed over by the main pass (RETAKE false) through the fix list
// and redone by the RETAKE pass, whose warps then all take the FP64 branch
// together.
template <class R, int STRAT> constexpr bool kRetakePass = sizeof(R) == 4 && (STRAT == 0 || STRAT == 2);

template <class R, int STRAT, bool B, bool RETAKE, bool QMC = false, class KER = nlq::KerConst>
__global__ void __launch_bounds__(EvCfg<R>::threads, EvCfg<R>::min_blocks) k_events(const __grid_constant__ AsmArgs A)
{
    extern __shared__ __align__(16) unsigned char evsm[];
    R *cb = reinterpret_cast<R *>(evsm) + nlq::CB_STRIDE * threadIdx.x;   // cell j at cb + j * CB_STRIDE * threads
    nlq::Stats st{0, 0, 0, 0, 0};
    const int64_t nu = 4 * (A.p1 - A.p0);
    const int n0 = A.nev[0], n1 = A.nev[1], n2 = A.nev[2], n3 = A.nev[3];
    const int nev = RETAKE ? A.nev[4] : n0 + n1 + n2 + n3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nev; i += gridDim.x * blockDim.x) {
        const int e = RETAKE ? A.fix[i] : i;
        // compact event index -> (class, index within the class)
        int c = 0, idx = e;
        if (idx >= n0) { idx -= n0; c = 1;
            if (idx >= n1) { idx -= n1; c = 2;
                if (idx >= n2) { idx -= n2; c = 3; } } }
        const int32_t u = A.evu[c * nu + idx];
        int64_t p;
        const Prob &P = prob_of_pair<B>(A, A.p0 + (u >> 2), p);
        const int q = u & 3;
        const int32_t T = P.pair_T[p], Tp = P.pair_tp[p];
        const int32_t o = P.outer_of[T];
        P3<R> v[4];
        P3<R> x;
        nlq::Strict sx;
        load_point_geometry<R>(P, P.tets[Tp], o, q, v, x, sx);
        const int inm = A.uinfo[u] & 15;
        // the record is built in shared memory and written out once
        R *out = reinterpret_cast<R *>(evsm) + 3 * nlq::CB_STRIDE * EvCfg<R>::threads + 17 * threadIdx.x;
        constexpr bool diag_inline = RETAKE || !kRetakePass<R, STRAT>;
        const R d2 = sizeof(R) == 4 ? (R)P.delta2f : (R)P.delta2;
        KER ker{};
        if constexpr (!KER::constant) ker = KER{(R)A.kc[0], (R)A.kc[1], (R)A.kc[2], (R)A.kc[3], d2};
        const bool deferred = nlq::event_moments<R, STRAT, diag_inline, false, QMC, KER>(
            v, x, d2, inm, A.nmc, A.rk, (uint32_t)T, (uint32_t)Tp,
            (uint32_t)q, out, st, (sizeof(R) == 4) ? &sx : nullptr, cb, nlq::CB_STRIDE * EvCfg<R>::threads,
            nlq::HullScratch<R>{reinterpret_cast<R *>(evsm) + threadIdx.x, EvCfg<R>::threads}, nullptr, A.hull_maxf,
            ker);
        if (deferred) {
            if constexpr (!RETAKE) A.fix[atomicAdd(&A.nev[4], 1)] = e;
        } else if constexpr (sizeof(R) == 4) {
            float4 *g = reinterpret_cast<float4 *>(A.Mq) + (MQ_STRIDE / 4) * (int64_t)u;
            g[0] = make_float4(out[0], out[1], out[2], out[3]);
            g[1] = make_float4(out[4], out[5], out[6], out[7]);
            g[2] = make_float4(out[8], out[9], out[10], out[11]);
            g[3] = make_float4(out[12], out[13], out[14], 0.f);
        } else {
            double2 *g = reinterpret_cast<double2 *>(A.Mq) + (MQ_STRIDE / 2) * (int64_t)u;
#pragma unroll
            for (int k = 0; k < 7; ++k) g[k] = make_double2(out[2 * k], out[2 * k + 1]);
            g[7] = make_double2(out[14], 0.0);
        }
    }
    __shared__ unsigned long long sstat[4];
    if (threadIdx.x < 4) sstat[threadIdx.x] = 0ULL;
    __syncthreads();
    if (!RETAKE && st.cut) atomicAdd(&sstat[0], (unsigned long long)st.cut);   // the main pass counted them
    if (st.mc) atomicAdd(&sstat[1], (unsigned long long)st.mc);
    if (st.acc) atomicAdd(&sstat[2], (unsigned long long)st.acc);
    if (st.fallback) atomicAdd(&sstat[3], (unsigned long long)st.fallback);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sstat[0]) atomicAdd(&A.stats[0], sstat[0]);
        if (sstat[1]) atomicAdd(&A.stats[2], sstat[1]);
        if (sstat[2]) atomicAdd(&A.stats[3], sstat[2]);
        if (sstat[3]) atomicAdd(&A.stats[4], sstat[3]);
    }
}

// ---------------------------------------------------------------------------
// K2b (FP32 approxcaps only): the events that K2 deferred are recomputed with
// the FP64 event code on global coordinates (same classification), and the
// moments stored in the event's FP32 record.
template <int STRAT, bool B>
__global__ void __launch_bounds__(64) k_events_fp64(const __grid_constant__ AsmArgs A)
{
    extern __shared__ __align__(16) unsigned char fsm[];   // hull scratch, threads interleaved
    nlq::Stats st{0, 0, 0, 0, 0};
    const int64_t nu = 4 * (A.p1 - A.p0);
    const int n0 = A.nev[0], n1 = A.nev[1], n2 = A.nev[2], nf = A.nev[4];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        const int e = A.fix[i];
        int c = 0, idx = e;
        if (idx >= n0) { idx -= n0; c = 1;
            if (idx >= n1) { idx -= n1; c = 2;
                if (idx >= n2) { idx -= n2; c = 3; } } }
        const int32_t u = A.evu[c * nu + idx];
        int64_t p;
        const Prob &P = prob_of_pair<B>(A, A.p0 + (u >> 2), p);
        const int q = u & 3;
        const int32_t T = P.pair_T[p], Tp = P.pair_tp[p];
        const int32_t o = P.outer_of[T];
        P3<double> v[4];
        P3<double> x;
        nlq::Strict sx;
        load_point_geometry<double>(P, P.tets[Tp], o, q, v, x, sx);
        const int inm = A.uinfo[u] & 15;
        double m15[15];
        nlq::event_moments<double, STRAT>(v, x, P.delta2, inm, A.nmc, A.rk, (uint32_t)T, (uint32_t)Tp, (uint32_t)q,
                                          m15, st, nullptr, nullptr, 0,
                                          nlq::HullScratch<double>{reinterpret_cast<double *>(fsm) + threadIdx.x, 64},
                                          nullptr, A.hull_maxf);
        float *out = reinterpret_cast<float *>(A.Mq) + MQ_STRIDE * (int64_t)u;
#pragma unroll
        for (int k = 0; k < 15; ++k) out[k] = (float)m15[k];
    }
    if (st.fallback) atomicAdd(&A.stats[4], (unsigned long long)st.fallback);
}


// ---------------------------------------------------------------------------
// K2' with a kernel shape phi (Sec. 2's gamma(x, y) = gamma phi(|x - y|)):
// the units whose T' is whole (every vertex inside, or an element-level
// strategy's full T') have no closed form any more; one thread per such unit
// takes the 4-point rule on T' with phi at the rule points and writes its
// record.  The cut units go through k_events with the same shape.
template <class R, bool B>
__global__ void __launch_bounds__(256) k_whole_shape(const __grid_constant__ AsmArgs A)
{
    const int64_t nu = 4 * (A.p1 - A.p0);
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x) {
        if (A.uinfo[u] != (15 | 0x10)) continue;
        int64_t p;
        const Prob &P = prob_of_pair<B>(A, A.p0 + (u >> 2), p);
        const int q = (int)(u & 3);
        const int32_t T = P.pair_T[p], Tp = P.pair_tp[p];
        const int32_t o = P.outer_of[T];
        P3<R> v[4];
        P3<R> x;
        nlq::Strict sx;
        load_point_geometry<R>(P, P.tets[Tp], o, q, v, x, sx);
        const R d2 = sizeof(R) == 4 ? (R)P.delta2f : (R)P.delta2;
        const nlq::KerShape<R> ker{(R)A.kc[0], (R)A.kc[1], (R)A.kc[2], (R)A.kc[3], d2};
        Mom<R> M;
        nlq::whole_moments<R>(v, x, (R)P.tet_vol[Tp], ker, M);
        if constexpr (sizeof(R) == 4) {
            float4 *g = reinterpret_cast<float4 *>(A.Mq) + (MQ_STRIDE / 4) * u;
            g[0] = make_float4(M.m0, M.m1[0], M.m1[1], M.m1[2]);
            g[1] = make_float4(M.m1[3], M.m2[0], M.m2[1], M.m2[2]);
            g[2] = make_float4(M.m2[3], M.m2[4], M.m2[5], M.m2[6]);
            g[3] = make_float4(M.m2[7], M.m2[8], M.m2[9], 0.f);
        } else {
            double2 *g = reinterpret_cast<double2 *>(A.Mq) + (MQ_STRIDE / 2) * u;
            g[0] = make_double2(M.m0, M.m1[0]); g[1] = make_double2(M.m1[1], M.m1[2]);
            g[2] = make_double2(M.m1[3], M.m2[0]); g[3] = make_double2(M.m2[1], M.m2[2]);
            g[4] = make_double2(M.m2[3], M.m2[4]); g[5] = make_double2(M.m2[5], M.m2[6]);
            g[6] = make_double2(M.m2[7], M.m2[8]); g[7] = make_double2(M.m2[9], 0.0);
        }
    }
}

// ---------------------------------------------------------------------------
// K3: one block per outer element T (persistent over the chunk's outer
// elements), one thread per pair: combine the four points of each pair into
// the staged T'T' moments, the TT sums and the cross strips:
//   TT   += c omega lambda(x_q) lambda(x_q)^T m0     (V_q summed per T)
//   TT'  -= c omega lambda(x_q) m1^T                  (strip rows of T's nodes)
//   T'T' += c omega m2                                 (staged per pair)
// with c = (gamma/2)|T|/4 and omega = 2 for collar elements T'.  Strips are
// accumulated by one warp per row in pair order (deterministic).
constexpr int NT = 128;
// per-pair stride of the 16 cross coefficients and their strip positions in
// shared memory: odd, so that neither the per-pair writes nor the row-wise
// reads of 8 pairs at a time pile up on a few banks
constexpr int XS = 17;

// SHAPE (FP32, a kernel shape, element-level strategies): the points at
// which T' is whole (info 15 | 0x10) take no FP32 record; their moments come
// from the kernel shape at T''s rule points in FP64 here, and enter the V_q
// sums and cross coefficients in double-float and the T'T' part through P.Dw
// in FP64, as the constant kernel's closed forms do.
template <class R, bool B, bool SHAPE = false>
__global__ void __launch_bounds__(NT) k_combine(const __grid_constant__ AsmArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int mr = A.max_row;
    int32_t *cols = reinterpret_cast<int32_t *>(smem);                                        // [4][mr]
    double *strip = reinterpret_cast<double *>(smem + sizeof(int32_t) * 4 * ((mr + 1) & ~1));  // [4][mr]
    // [NT][XS] cross coefficients: R for FP64, double-float for FP32 (8 bytes either way)
    double *Xs = strip + 4 * mr;
    int32_t *offs = reinterpret_cast<int32_t *>(Xs + NT * XS);                                 // [NT][XS]
    double *wsc = reinterpret_cast<double *>(offs + NT * XS);                                  // [NT]
    double *red = wsc + NT;                                                                    // [NT/32][4]
    __shared__ int lens[4];
    __shared__ unsigned long long sin_;
    constexpr bool F32 = sizeof(R) == 4;
    static_assert(sizeof(DF) == sizeof(double), "strip and weight slots hold a double or a double-float");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long inside = 0;

    for (int64_t og = A.o0 + blockIdx.x; og < A.o1; og += gridDim.x) {
        int64_t o;
        const Prob &P = prob_of_outer<B>(A, og, o);
        const int32_t T = P.outer_ids[o];
        const int4 eT = P.tets[T];
        const int nodeT[4] = {eT.x, eT.y, eT.z, eT.w};
        if (tid < 4) lens[tid] = (int)(P.rowptr[nodeT[tid] + 1] - P.rowptr[nodeT[tid]]);
        __syncthreads();
        for (int i = 0; i < 4; ++i) {
            const int64_t rb = P.rowptr[nodeT[i]];
            for (int c = tid; c < lens[i]; c += NT) {
                cols[i * mr + c] = P.col[rb + c];
                strip[i * mr + c] = 0.0;     // also DF{0, 0} for the FP32 path
            }
        }
        const double cT = P.half_gamma * (P.tet_vol[T] * 0.25);
        const DF cTf = df_from(cT);
        double vq[4] = {0.0, 0.0, 0.0, 0.0};
        DF vqf[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        __syncthreads();
        const int64_t pb = P.pair_ptr[o], pe = P.pair_ptr[o + 1];
        for (int64_t base = pb; base < pe; base += NT) {
            const int cnt = (int)((pe - base) < (int64_t)NT ? (pe - base) : (int64_t)NT);
            const int64_t p = base + tid;
            if (tid < cnt) {
                const int32_t Tp = P.pair_tp[p];
                const int4 eP = P.tets[Tp];
                const int nodeP[4] = {eP.x, eP.y, eP.z, eP.w};
                const double omega = P.in_omega[Tp] ? 1.0 : 2.0;
                const R volTp = (R)P.tet_vol[Tp];
                R Y[4][4], V[4], Dp[10];
#pragma unroll
                for (int k = 0; k < 10; ++k) Dp[k] = R(0);
                const int64_t u0 = 4 * (P.pair_base + p - A.p0);
                // FP32: points where T' is whole enter in double (their moments
                // are closed forms of |T'|), the others from their FP32 records
                int fullmask = 0, wmask = 0;
                // the pair's 4 units: 4 info bytes in one load (u0 is a multiple
                // of 4)
                const uint32_t info4 = *reinterpret_cast<const uint32_t *>(A.uinfo + u0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint8_t info = (uint8_t)(info4 >> (8 * q));
                    Mom<R> M;
                    bool wshape = false;
                    if constexpr (SHAPE) wshape = info == (15 | 0x10);
                    if (wshape) {
                        nlq::mom_zero(M);
                        wmask |= 1 << q;
                        inside++;
                    } else if ((info & 15) == 15 && !(info & 0x10)) {
                        if constexpr (F32) {
                            nlq::mom_zero(M);
                            fullmask |= 1 << q;
                        } else {
                            nlq::closed_form_inside(M, volTp);
                        }
                        inside++;
                    } else if (info & 0x10) {
                        // (with a kernel shape, a whole T' has a record too)
                        if ((info & 15) == 15) inside++;
                        // the unit's record (records are stored by unit: the
                        // pair's four are contiguous)
                        const int64_t ev = u0 + q;
                        R mq[MQ_STRIDE];
                        if constexpr (F32) {
                            const float4 *m4 = reinterpret_cast<const float4 *>(A.Mq) + (MQ_STRIDE / 4) * ev;
#pragma unroll
                            for (int k = 0; k < MQ_STRIDE / 4; ++k) {
                                const float4 t4 = m4[k];
                                mq[4 * k] = t4.x; mq[4 * k + 1] = t4.y; mq[4 * k + 2] = t4.z; mq[4 * k + 3] = t4.w;
                            }
                        } else {
                            const double2 *m2 = reinterpret_cast<const double2 *>(A.Mq) + (MQ_STRIDE / 2) * ev;
#pragma unroll
                            for (int k = 0; k < MQ_STRIDE / 2; ++k) {
                                const double2 t2 = m2[k];
                                mq[2 * k] = t2.x; mq[2 * k + 1] = t2.y;
                            }
                        }
                        M.m0 = mq[0];
#pragma unroll
                        for (int k = 0; k < 4; ++k) M.m1[k] = mq[1 + k];
#pragma unroll
                        for (int k = 0; k < 10; ++k) M.m2[k] = mq[5 + k];
                    } else {
                        nlq::mom_zero(M);
                    }
                    V[q] = M.m0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) Y[q][k] = M.m1[k];
#pragma unroll
                    for (int k = 0; k < 10; ++k) Dp[k] += M.m2[k];
                }
                R *Dst = reinterpret_cast<R *>(P.D) + 10 * p;
#pragma unroll
                for (int k = 0; k < 10; ++k) Dst[k] = Dp[k];
                if constexpr (F32) {
                    const int nfull = __popc(fullmask);
                    P.nfull[p] = (uint8_t)nfull;
                    // kernel shapes: phi at T''s rule points for its whole points
                    // (FP64), the unit's moments being (|T'|/4) sums of phi
                    // times the rule's barycentrics (a on the own vertex, b else)
                    double wphi[4][4], wS[4];
                    const double V4 = P.tet_vol[Tp] * 0.25;
                    const double wqa = 0x1.2bbae2a27f931p-1, wqb = 0x1.1b06d1d200913p-3, wqd = wqa - wqb;
                    if constexpr (SHAPE) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            wS[q] = 0.0;
#pragma unroll
                            for (int k = 0; k < 4; ++k) wphi[q][k] = 0.0;
                        }
                        if (wmask) {
                            const double4 g0 = P.verts[eP.x], g1 = P.verts[eP.y], g2 = P.verts[eP.z], g3 = P.verts[eP.w];
                            const double sx = (g0.x + g1.x) + (g2.x + g3.x), sy = (g0.y + g1.y) + (g2.y + g3.y),
                                         sz = (g0.z + g1.z) + (g2.z + g3.z);
                            const double4 gk[4] = {g0, g1, g2, g3};
                            const double *xo = P.xq + 12 * o;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                if (!((wmask >> q) & 1)) continue;
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const double wx = wqb * sx + wqd * gk[k].x - xo[3 * q];
                                    const double wy = wqb * sy + wqd * gk[k].y - xo[3 * q + 1];
                                    const double wz = wqb * sz + wqd * gk[k].z - xo[3 * q + 2];
                                    double ss = ((wx * wx + wy * wy) + wz * wz) / P.delta2;
                                    ss = ss < 1.0 ? ss : 1.0;
                                    const double ph = A.kc[0] + ss * (A.kc[1] + ss * (A.kc[2] + ss * A.kc[3]));
                                    wphi[q][k] = ph;
                                    wS[q] += ph;
                                }
                            }
                        }
                        // T'T' part: sum over the whole points of
                        // (|T'|/4) (b^2 S + b d (phi_a + phi_b) + [a = b] d^2 phi_a)
                        double *dw = P.Dw + 10 * p;
                        int t = 0;
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int b = a; b < 4; ++b) {
                                double v = 0.0;
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    v += V4 * ((wqb * wqb) * wS[q] + (wqb * wqd) * (wphi[q][a] + wphi[q][b]) +
                                               (a == b ? (wqd * wqd) * wphi[q][a] : 0.0));
                                dw[t++] = v;
                            }
                    }
                    // |T'| as float hi + lo; omega is 1 or 2 (exact scaling)
                    const float2 vhl = P.vol_hl[Tp];
                    const float omf = P.in_omega[Tp] ? 1.f : 2.f;
                    const DF wV{omf * vhl.x, omf * vhl.y};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        vqf[q] = df_add(vqf[q], DF{omf * (float)V[q], 0.f});
                        if ((fullmask >> q) & 1) vqf[q] = df_add(vqf[q], wV);
                        if constexpr (SHAPE) {
                            if ((wmask >> q) & 1) vqf[q] = df_add(vqf[q], df_from((double)omf * (V4 * wS[q])));
                        }
                    }
                    // weights of the 4-point rule as float hi + lo
                    const DF qa = df_const(0x1.2bbae2a27f931p-1), qb = df_const(0x1.1b06d1d200913p-3);
                    const DF v4{0.25f * vhl.x, 0.25f * vhl.y};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        // whole-T' points: sum over them of lambda_i(x_q) |T'| / 4
                        const int own = (fullmask >> i) & 1;
                        DF xc{0.f, 0.f};
                        if (nfull) {
                            // own x a + (nfull - own) x b, products exact by fused multiply-add
                            const DF s = df_add(own ? qa : DF{0.f, 0.f}, df_mul(qb, (float)(nfull - own)));
                            xc = df_mul2(v4, s);
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float ev = ((qlam<float>(i, 0) * (float)Y[0][k] + qlam<float>(i, 1) * (float)Y[1][k]) +
                                              qlam<float>(i, 2) * (float)Y[2][k]) + qlam<float>(i, 3) * (float)Y[3][k];
                            DF xs = df_add(xc, DF{ev, 0.f});
                            if constexpr (SHAPE) {
                                if (wmask) {
                                    // the whole points' first moments, (|T'|/4)(b S + d phi_k)
                                    double xw = 0.0;
#pragma unroll
                                    for (int q = 0; q < 4; ++q)
                                        xw += qlam<double>(i, q) * (V4 * (wqb * wS[q] + wqd * wphi[q][k]));
                                    xs = df_add(xs, df_from(xw));
                                }
                            }
                            reinterpret_cast<DF *>(Xs)[tid * XS + 4 * i + k] = xs;
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) vq[q] += omega * (double)V[q];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            R sum = ((qlam<R>(i, 0) * Y[0][k] + qlam<R>(i, 1) * Y[1][k]) + qlam<R>(i, 2) * Y[2][k]) +
                                    qlam<R>(i, 3) * Y[3][k];
                            Xs[tid * XS + 4 * i + k] = (double)sum;
                        }
                }
                // positions of T''s nodes in the rows of T's nodes (present
                // in every one of them): branch-free lower bounds, the four
                // keys of a row in lockstep (the rows are the block's, so the
                // warp does not diverge)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int32_t *row = cols + i * mr;
                    int b[4] = {0, 0, 0, 0};
                    for (int n = lens[i]; n > 1;) {
                        const int half = n >> 1;
#pragma unroll
                        for (int k = 0; k < 4; ++k) b[k] = (row[b[k] + half] < nodeP[k]) ? b[k] + half : b[k];
                        n -= half;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) offs[tid * XS + 4 * i + k] = b[k] + (row[b[k]] < nodeP[k] ? 1 : 0);
                }
                // the weight -omega c_T: FP32 path in double-float (omega = 1
                // or 2 scales exactly; no FP64 work per pair)
                if constexpr (F32) {
                    const float omf = P.in_omega[Tp] ? -1.f : -2.f;
                    reinterpret_cast<DF *>(wsc)[tid] = DF{omf * cTf.hi, omf * cTf.lo};
                } else {
                    wsc[tid] = -(omega * cT);
                }
            }
            __syncthreads();
            {
                // warp i adds row i's contributions of 8 pairs at a time (lane =
                // 4 * pair + k); lanes that hit the same column are summed by
                // the lowest of them in ascending lane order, so the sum order
                // is fixed by the pair order alone
                const int i = warp;
                for (int g0 = 0; g0 < cnt; g0 += 8) {
                    const int t = g0 + (lane >> 2), k = lane & 3;
                    const bool act = t < cnt;
                    const int c = act ? offs[t * XS + 4 * i + k] : -1 - lane;
                    const unsigned peers = __match_any_sync(0xffffffffu, c);
                    const int leader = __ffs(peers) - 1;
                    const int maxn = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(peers));
                    unsigned rest = (lane == leader) ? (peers & (peers - 1u)) : 0u;
                    if constexpr (F32) {
                        const DF v = act ? df_mul2(reinterpret_cast<const DF *>(wsc)[t],
                                                   reinterpret_cast<const DF *>(Xs)[t * XS + 4 * i + k])
                                         : DF{0.f, 0.f};
                        DF sum = v;
                        for (int j = 1; j < maxn; ++j) {
                            const int src = rest ? __ffs(rest) - 1 : lane;
                            const float wh = __shfl_sync(0xffffffffu, v.hi, src);
                            const float wl = __shfl_sync(0xffffffffu, v.lo, src);
                            if (rest) { sum = df_add(sum, DF{wh, wl}); rest &= rest - 1u; }
                        }
                        DF *sp = reinterpret_cast<DF *>(strip);
                        if (act && lane == leader) sp[i * mr + c] = df_add(sp[i * mr + c], sum);
                    } else {
                        const double v = act ? wsc[t] * Xs[t * XS + 4 * i + k] : 0.0;
                        double sum = v;
                        for (int j = 1; j < maxn; ++j) {
                            const int src = rest ? __ffs(rest) - 1 : lane;
                            const double w = __shfl_sync(0xffffffffu, v, src);
                            if (rest) { sum += w; rest &= rest - 1u; }
                        }
                        if (act && lane == leader) strip[i * mr + c] += sum;
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (F32) {
                DF sum = vqf[q];
                for (int off = 16; off > 0; off >>= 1)
                    sum = df_add(sum, DF{__shfl_xor_sync(0xffffffffu, sum.hi, off),
                                         __shfl_xor_sync(0xffffffffu, sum.lo, off)});
                if (lane == 0) red[warp * 4 + q] = df_to(sum);
            } else {
                double sum = vq[q];
                for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
                if (lane == 0) red[warp * 4 + q] = sum;
            }
        }
        __syncthreads();
        if (tid < 10) {
            double V[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) V[q] = (red[0 * 4 + q] + red[1 * 4 + q]) + (red[2 * 4 + q] + red[3 * 4 + q]);
            const int ia[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
            const int ib[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
            const int i = ia[tid], j = ib[tid];
            double sum = 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q) sum += qlam<double>(i, q) * qlam<double>(j, q) * V[q];
            P.TT[10 * o + tid] = cT * sum;
        }
        for (int i = 0; i < 4; ++i) {
            const int64_t so = P.strip_off[4 * o + i];
            for (int c = tid; c < lens[i]; c += NT)
                P.strips[so + c] = F32 ? df_to(reinterpret_cast<const DF *>(strip)[i * mr + c]) : strip[i * mr + c];
        }
        __syncthreads();
    }
    if (tid == 0) sin_ = 0ULL;
    __syncthreads();
    if (inside) atomicAdd(&sin_, inside);
    __syncthreads();
    if (tid == 0 && sin_) atomicAdd(&A.stats[1], sin_);
}

inline size_t combine_smem_bytes(int max_row, size_t real_size)
{
    size_t b = sizeof(int32_t) * 4 * (size_t)((max_row + 1) & ~1);
    b += sizeof(double) * 4 * (size_t)max_row;
    b += sizeof(double) * NT * XS;     // cross coefficients (double or double-float)
    (void)real_size;
    b += sizeof(int32_t) * NT * XS;
    b += sizeof(double) * NT;
    b += sizeof(double) * (NT / 32) * 4;
    return b;
}

// Work arrays of one chunk (reused by every chunk of a launch).
template <class R, int STRAT>
void alloc_work(AsmArgs &A, Scratch &sc, int64_t max_units)
{
    constexpr bool kDefer = sizeof(R) == 4 && STRAT == 1;
    A.uinfo = sc.get<uint8_t>(max_units);
    A.evu = sc.get<int32_t>(4 * max_units);
    A.nev = sc.get<int>(5);
    A.fix = (kDefer || kRetakePass<R, STRAT>) ? sc.get<int32_t>(max_units) : nullptr;
    A.Mq = (void *)sc.get<R>(MQ_STRIDE * max_units);
}

// The three quadrature kernels over every chunk, stream-ordered, no host
// synchronisation (capturable in a CUDA graph).  ev, when given, receives 4
// events per chunk around the kernels.
template <class R, int STRAT, bool B>
void launch_chunks(AsmArgs A, const std::vector<int64_t> &gptr, const std::vector<std::pair<int64_t, int64_t>> &chunks,
                   const Shape &sh, cudaStream_t s, cudaEvent_t *ev)
{
    constexpr bool kDefer = sizeof(R) == 4 && STRAT == 1;
    const size_t smem = combine_smem_bytes(A.max_row, sizeof(R));
    NL_REQUIRE(smem <= 220 * 1024, "rows of %d columns need %zu bytes of shared memory", A.max_row, smem);
    // kernel shapes, FP32, element-level strategies (every unit is a whole
    // T'): k_combine takes the whole points itself in FP64; otherwise they
    // come from k_whole_shape's records, and the cut units' FP32 records set
    // the accuracy anyway
    constexpr bool kShapeCombine = sizeof(R) == 4 && !B && STRAT >= 3;
    void (*k3)(const AsmArgs) = k_combine<R, B>;
    if constexpr (kShapeCombine) {
        if (A.kpoly) k3 = k_combine<R, B, true>;
    }
    // the attribute is per function and process-wide: always the same limit,
    // so concurrent launches of other sizes (other threads) never lower it
    NL_CUDA(cudaFuncSetAttribute(k3, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    int per_sm = 0;
    NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3, NT, smem));
    per_sm = per_sm < 1 ? 1 : per_sm;
    int ev_per_sm = 0;
    constexpr int ET = EvCfg<R>::threads;
    constexpr size_t ESM = EvCfg<R>::smem;
    // the event kernels (main pass, retake pass) of the group's sampler
    void (*ev_main)(const AsmArgs) = nullptr;
    void (*ev_retake)(const AsmArgs) = nullptr;
    if constexpr (STRAT <= 2) {
        ev_main = k_events<R, STRAT, B, false>;
        ev_retake = k_events<R, STRAT, B, true>;
        if constexpr (STRAT == 2) {
            if (A.qmc) { ev_main = k_events<R, 2, B, false, true>; ev_retake = k_events<R, 2, B, true, true>; }
        }
        if constexpr (!B && STRAT != 1) {
            if (A.kpoly) {
                using KS = nlq::KerShape<R>;
                ev_main = k_events<R, STRAT, B, false, false, KS>;
                ev_retake = k_events<R, STRAT, B, true, false, KS>;
                if constexpr (STRAT == 2) {
                    if (A.qmc) { ev_main = k_events<R, 2, B, false, true, KS>; ev_retake = k_events<R, 2, B, true, true, KS>; }
                }
            }
        }
        NL_CUDA(cudaFuncSetAttribute(ev_main, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ESM));
        if constexpr (kRetakePass<R, STRAT>)
            NL_CUDA(cudaFuncSetAttribute(ev_retake, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ESM));
        NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ev_per_sm, ev_main, ET, ESM));
    }
    ev_per_sm = ev_per_sm < 1 ? 1 : ev_per_sm;
    if (sh.events_blocks_per_sm > 0) ev_per_sm = std::min(ev_per_sm, sh.events_blocks_per_sm);
    // kernel shapes (single problems, not approxcaps): the event kernels with
    // the shape, and k_whole_shape for the whole T' units
    const bool shape = !B && STRAT != 1 && A.kpoly;
    (void)shape;
    const int sms = nl_num_sms();
    const int ct = sh.classify_threads;
    size_t ci = 0;
    for (auto &c : chunks) {
        A.o0 = c.first; A.o1 = c.second;
        A.p0 = gptr[c.first]; A.p1 = gptr[c.second];
        const int64_t nu = 4 * (A.p1 - A.p0);
        NL_CUDA(cudaMemsetAsync(A.nev, 0, 5 * sizeof(int), s));
        unsigned g1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nl_cdiv<int64_t>(nu, ct), (int64_t)sms * (8192 / ct)));
        if (ev) NL_CUDA(cudaEventRecord(ev[4 * ci], s));
        { k_classify<R, STRAT, B><<<g1, ct, 0, s>>>(A); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        if (ev) NL_CUDA(cudaEventRecord(ev[4 * ci + 1], s));
        // enough resident threads for the largest possible event count; the
        // kernel reads the actual count from device memory
        unsigned g2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nl_cdiv<int64_t>(nu, ET), (int64_t)sms * ev_per_sm));
        if constexpr (!B && !kShapeCombine) {
            if (shape) {
                const unsigned gw = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nl_cdiv<int64_t>(nu, 256),
                                                                                     (int64_t)sms * 8));
                { k_whole_shape<R, B><<<gw, 256, 0, s>>>(A); nl_count_launch(); }
                NL_CHECK_LAUNCH();
            }
        }
        if constexpr (STRAT <= 2) {
            { ev_main<<<g2, ET, ESM, s>>>(A); nl_count_launch(); }
            NL_CHECK_LAUNCH();
        }
        if constexpr (kDefer) {
            { k_events_fp64<STRAT, B><<<(unsigned)(2 * sms), 64, sizeof(double) * 64 * nlq::HULL_SCRATCH, s>>>(A);
              nl_count_launch(); }
            NL_CHECK_LAUNCH();
        }
        if constexpr (kRetakePass<R, STRAT>) {
            // the handed-over events (a few per cent; the kernel reads their
            // count from device memory); full occupancy, as their FP64 work is
            // latency-bound
            { ev_retake<<<(unsigned)(sms * ev_per_sm), ET, ESM, s>>>(A); nl_count_launch(); }
            NL_CHECK_LAUNCH();
        }
        if (ev) NL_CUDA(cudaEventRecord(ev[4 * ci + 2], s));
        int64_t no = A.o1 - A.o0;
        unsigned g3 = (unsigned)std::min<int64_t>(no, (int64_t)sms * per_sm);
        { k3<<<g3, NT, smem, s>>>(A); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        if (ev) NL_CUDA(cudaEventRecord(ev[4 * ci + 3], s));
        ++ci;
    }
}

template <class R, int STRAT>
void run_single(nl_system *sys, AsmArgs &A)
{
    nl_pairs *P = sys->pairs;
    nl_mesh *m = P->mesh;
    cudaStream_t s = sys->arena.stream();
    std::vector<int64_t> hp(m->n_outer + 1);
    NL_CUDA(cudaMemcpyAsync(hp.data(), P->pair_ptr, sizeof(int64_t) * (m->n_outer + 1), cudaMemcpyDeviceToHost, s));
    NL_CUDA(cudaStreamSynchronize(s));
    int64_t max_units = 0;
    auto chunks = plan_chunks(hp, kUnitsPerChunk, &max_units);
    Scratch sc(&sys->arena);
    alloc_work<R, STRAT>(A, sc, max_units);
    std::vector<cudaEvent_t> ev(4 * chunks.size());
    for (auto &e : ev) NL_CUDA(cudaEventCreate(&e));
    launch_chunks<R, STRAT, false>(A, hp, chunks, Shape(), s, ev.data());
    NL_CUDA(cudaStreamSynchronize(s));
    double t[3] = {0.0, 0.0, 0.0};
    for (size_t k = 0; k < chunks.size(); ++k)
        for (int j = 0; j < 3; ++j) {
            float ms = 0.f;
            NL_CUDA(cudaEventElapsedTime(&ms, ev[4 * k + j], ev[4 * k + j + 1]));
            t[j] += ms;
        }
    for (auto &e : ev) cudaEventDestroy(e);
    sys->stats.classify_ms = t[0];
    sys->stats.events_ms = t[1];
    sys->stats.combine_ms = t[2];
}


template <class R>
void launch_assemble(nl_system *sys, void *D, double *strips, double *TT, uint8_t *nfull, unsigned long long *stats)
{
    AsmArgs A;
    memset(&A, 0, sizeof(A));
    A.self = make_prob(sys, D, strips, TT, nfull);
    init_group_args(A, sys->opts, stats, sys->pairs->max_row);
    switch (sys->opts.strategy) {
    case NL_NOCAPS: run_single<R, 0>(sys, A); break;
    case NL_APPROXCAPS: run_single<R, 1>(sys, A); break;
    case NL_FULLCAPS:
    case NL_FULLCAPS_QMC: run_single<R, 2>(sys, A); break;
    case NL_BARYCENTER: run_single<R, 3>(sys, A); break;
    case NL_OVERLAP: run_single<R, 4>(sys, A); break;
    default: run_single<R, 5>(sys, A); break;
    }
}

template <class R>
void launch_group(const BatchGroup &g, const Shape &sh, cudaStream_t s)
{
    int64_t mu = 0;
    auto chunks = plan_chunks(g.gptr, sh.units_per_chunk, &mu);
    switch (g.strategy) {
    case NL_NOCAPS: launch_chunks<R, 0, true>(g.A, g.gptr, chunks, sh, s, nullptr); break;
    case NL_APPROXCAPS: launch_chunks<R, 1, true>(g.A, g.gptr, chunks, sh, s, nullptr); break;
    case NL_FULLCAPS:
    case NL_FULLCAPS_QMC: launch_chunks<R, 2, true>(g.A, g.gptr, chunks, sh, s, nullptr); break;
    case NL_BARYCENTER: launch_chunks<R, 3, true>(g.A, g.gptr, chunks, sh, s, nullptr); break;
    case NL_OVERLAP: launch_chunks<R, 4, true>(g.A, g.gptr, chunks, sh, s, nullptr); break;
    default: launch_chunks<R, 5, true>(g.A, g.gptr, chunks, sh, s, nullptr); break;
    }
}

// Work arrays for the largest chunk any candidate shape can form.
template <class R>
void alloc_group_work(BatchGroup &g, DevArena &arena, int64_t max_units, std::vector<void *> &owned)
{
    Scratch sc(&arena);
    switch (g.strategy) {
    case NL_NOCAPS: alloc_work<R, 0>(g.A, sc, max_units); break;
    case NL_APPROXCAPS: alloc_work<R, 1>(g.A, sc, max_units); break;
    default: alloc_work<R, 2>(g.A, sc, max_units); break;
    }
    owned.insert(owned.end(), sc.mine.begin(), sc.mine.end());
    sc.mine.clear();    // kept by the batch
}

}  // namespace nla

namespace nla {

// Diagnostic kernel: moments of one (T', x) case per thread, with the same
// device code (and, per translation unit, the same compiler flags) as the
// assembly kernel.  For float, coordinates are made relative to x as
// double-float differences exactly as in the assembly.
struct RoundKeys {
    uint32_t k[20];
};

template <class R, int STRAT, bool REC = false, bool QMC = false>
__global__ void k_probe(const double *__restrict__ tv, const double4 *__restrict__ tv4, const double *__restrict__ xs,
                        const uint32_t *__restrict__ ids, int64_t n, double delta2, int nmc,
                        const __grid_constant__ RoundKeys rk, double *out, int *defer, double *rec = nullptr,
                        int *nrec = nullptr)
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
    sx.verts = tv4;
    sx.e = make_int4((int)(4 * c), (int)(4 * c + 1), (int)(4 * c + 2), (int)(4 * c + 3));
    sx.x = xs + 3 * c;
    sx.d2 = delta2;
    // 16-byte aligned: the sampler reads it with 16-byte loads; also the
    // approxcaps hull's scratch (that strategy does not sample)
    __align__(16) R cb[3 * nlq::CB_STRIDE];
    static_assert(3 * nlq::CB_STRIDE >= nlq::HULL_SCRATCH, "hull scratch");
    const int d = nlq::point_moments<R, STRAT, REC, QMC>(v, xx, (R)delta2, (R)vol, nmc, rk.k, ids[3 * c], ids[3 * c + 1],
                                                    ids[3 * c + 2], M, st, sizeof(R) == 4 ? &sx : nullptr, cb,
                                                    nlq::CB_STRIDE, nlq::HullScratch<R>{cb, 1},
                                                    REC ? rec + (int64_t)5 * nmc * c : nullptr,
                                                    REC ? nrec + c : nullptr);
    defer[c] = d;
    if (d) return;
    out[15 * c] = (double)M.m0;
    for (int k = 0; k < 4; ++k) out[15 * c + 1 + k] = (double)M.m1[k];
    for (int k = 0; k < 10; ++k) out[15 * c + 5 + k] = (double)M.m2[k];
}

// The deferred FP32 cases (defer[c] = classification + 1), recomputed with
// the FP64 event code and rounded through float as in the assembly's records.
template <int STRAT>
__global__ void k_probe_fp64(const double *__restrict__ tv, const double *__restrict__ xs,
                             const uint32_t *__restrict__ ids, int64_t n, double delta2, int nmc,
                             const __grid_constant__ RoundKeys rk, double *out, const int *defer)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || defer[c] == 0) return;
    const double *t = tv + 12 * c;
    P3<double> v[4];
    for (int k = 0; k < 4; ++k) v[k] = nlq::mk3<double>(t[3 * k], t[3 * k + 1], t[3 * k + 2]);
    P3<double> x = nlq::mk3<double>(xs[3 * c], xs[3 * c + 1], xs[3 * c + 2]);
    nlq::Stats st{0, 0, 0, 0, 0};
    double m15[15], hb[nlq::HULL_SCRATCH];
    nlq::event_moments<double, STRAT>(v, x, delta2, defer[c] - 1, nmc, rk.k, ids[3 * c], ids[3 * c + 1],
                                      ids[3 * c + 2], m15, st, nullptr, nullptr, 0, nlq::HullScratch<double>{hb, 1});
    for (int k = 0; k < 15; ++k) out[15 * c + k] = (double)(float)m15[k];
}

// The fullcaps Monte Carlo samples of each case (REC instantiation of the
// probe kernel): rec[c][k][5] = (cap cell, accepted, y), nrec[c] = samples
// drawn (0 without a cap or for a deferred case).
template <class R>
void launch_probe_samples(const double *tv, const double4 *tv4, const double *xs, const uint32_t *ids, int64_t n,
                          double delta2, int nmc, uint64_t seed, int qmc, double *out, int *defer, double *rec,
                          int *nrec)
{
    RoundKeys key;
    philox_round_keys(seed, key.k);
    unsigned blocks = (unsigned)((n + 127) / 128);
    if (qmc) k_probe<R, 2, true, true><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, nmc, key, out, defer, rec, nrec);
    else k_probe<R, 2, true><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, nmc, key, out, defer, rec, nrec);
    nl_count_launch();
    NL_CHECK_LAUNCH();
}

template <class R>
void launch_probe(const double *tv, const double4 *tv4, const double *xs, const uint32_t *ids, int64_t n,
                  double delta2, int strategy, int nmc, uint64_t seed, double *out, int *defer)
{
    RoundKeys key;
    philox_round_keys(seed, key.k);
    unsigned blocks = (unsigned)((n + 127) / 128);
    if (strategy == NL_NOCAPS) { k_probe<R, 0><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, 0, key, out, defer); nl_count_launch(); }
    else if (strategy == NL_APPROXCAPS) { k_probe<R, 1><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, 0, key, out, defer); nl_count_launch(); }
    else if (strategy == NL_FULLCAPS) { k_probe<R, 2><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, nmc, key, out, defer); nl_count_launch(); }
    else if (strategy == NL_FULLCAPS_QMC) { k_probe<R, 2, false, true><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, nmc, key, out, defer); nl_count_launch(); }
    else if (strategy == NL_BARYCENTER) { k_probe<R, 3><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, 0, key, out, defer); nl_count_launch(); }
    else if (strategy == NL_OVERLAP) { k_probe<R, 4><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, 0, key, out, defer); nl_count_launch(); }
    else { k_probe<R, 5><<<blocks, 128>>>(tv, tv4, xs, ids, n, delta2, 0, key, out, defer); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    if (sizeof(R) == 4 && strategy == NL_APPROXCAPS) {
        { k_probe_fp64<1><<<blocks, 64 * 2>>>(tv, xs, ids, n, delta2, 0, key, out, defer); nl_count_launch(); }
        NL_CHECK_LAUNCH();
    }
}

}  // namespace nla
