// Conjugate gradients on A u = b (Alg. 5, last line) with a CSR SpMV.
// FP64 mode: all vectors and values in FP64.  Mixed mode: iterative
// refinement with FP64 residuals r = b - A u and FP64 updates, the correction
// solved by CG on the FP32 copy of A with FP32 vectors; dot products are
// accumulated in FP64 in both modes.  Reductions use a fixed grid and a
// fixed combination order, so results are bitwise reproducible.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>

#include "nl_internal.h"

namespace {

struct CgState {
    double rr, pq, alpha, beta, tol2;
    int done, it;
    unsigned int ticket;     // blocks of the current reduction that have written their partial
    unsigned int bar_count;  // grid barrier of the single-launch CG: arrivals,
    unsigned int bar_gen;    // generation,
    int bar_err;             // set when a wait gave up (bounded spin)
};

constexpr int RB = 256;   // threads per block in reductions

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    __syncthreads();
    return s;   // valid in thread 0
}

// q = A p (warp per row) and per-block partial of p.q
// Sum of the nb block partials in a fixed order (lane l takes l, l+32, ...,
// then a fixed butterfly); called by one full warp.
__device__ __forceinline__ double warp_sum_parts(const double *part, int nb)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < nb; i += 32) s += __ldcg(part + i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// The last block to finish a reduction (the others have written their
// partials and passed a fence) sums the partials; returns true in that
// block's first warp.
__device__ __forceinline__ bool last_block(CgState *st)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    return last && threadIdx.x < 32;
}

// One row of A p on the padded rows, by the L lanes sub = 0..L-1 of a lane
// group (each lane's partial sum; the caller adds the L): FP32 values as
// float4 with int4 columns, FP64 values as double2 with int2 columns, and
// four 16-byte chunks of each lane loaded before their gathers, so that a row
// of several hundred entries costs a few memory round trips, not one per 32
// entries.  Pads hold value 0 and the row's own column.
template <class VT, class XT, int L = 8>
__device__ __forceinline__ VT pad_row(const int64_t *__restrict__ rp4, const int32_t *__restrict__ cp,
                                      const VT *__restrict__ vp, const XT *__restrict__ p, int64_t r, int sub)
{
    constexpr int U = 4;
    VT s = VT(0);
    if constexpr (sizeof(VT) == 4) {
        const int4 *c4 = reinterpret_cast<const int4 *>(cp);
        const float4 *v4 = reinterpret_cast<const float4 *>(vp);
        const int64_t e0 = rp4[r], e1 = rp4[r + 1];
        for (int64_t e = e0 + sub; e < e1; e += L * U) {
            float4 v[U];
            int4 c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t ee = e + L * u;
                if (ee < e1) { v[u] = __ldcs(v4 + ee); c[u] = __ldcs(c4 + ee); }
                else { v[u] = make_float4(0.f, 0.f, 0.f, 0.f); c[u] = make_int4(0, 0, 0, 0); }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                s += v[u].x * (VT)__ldg(p + c[u].x);
                s += v[u].y * (VT)__ldg(p + c[u].y);
                s += v[u].z * (VT)__ldg(p + c[u].z);
                s += v[u].w * (VT)__ldg(p + c[u].w);
            }
        }
    } else {
        const int2 *c2 = reinterpret_cast<const int2 *>(cp);
        const double2 *v2 = reinterpret_cast<const double2 *>(vp);
        const int64_t e0 = 2 * rp4[r], e1 = 2 * rp4[r + 1];
        for (int64_t e = e0 + sub; e < e1; e += L * U) {
            double2 v[U];
            int2 c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t ee = e + L * u;
                if (ee < e1) { v[u] = __ldcs(v2 + ee); c[u] = __ldcs(c2 + ee); }
                else { v[u] = make_double2(0.0, 0.0); c[u] = make_int2(0, 0); }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                s += v[u].x * (VT)__ldg(p + c[u].x);
                s += v[u].y * (VT)__ldg(p + c[u].y);
            }
        }
    }
    return s;
}

// q = A p on the padded rows (spmv_lanes<VT> lanes per row: 16 for FP32
// values, 8 for FP64) with the per-block partials of p.q; in the CG the last
// block forms alpha.  Every warp walks the same number of row groups (rows
// beyond n are skipped), so the lane-group sums can use full-warp shuffles.
// The grid is the resident blocks at most (spmv_blocks): each row group walks
// a few rows with all of them in flight, and no second wave of blocks trails
// the first.
template <class VT> __host__ __device__ constexpr int spmv_lanes() { return sizeof(VT) == 4 ? 16 : 8; }

template <class VT, class XT>
__global__ void __launch_bounds__(RB) k_spmv_dot_pad(const int64_t *__restrict__ rp4, const int32_t *__restrict__ cp,
                                                     const VT *__restrict__ vp, const XT *__restrict__ p, XT *q,
                                                     int64_t n, double *part, CgState *st)
{
    constexpr int L = spmv_lanes<VT>();
    __shared__ double sh[RB / 32];
    if (st && st->done) return;
    const int lane = threadIdx.x & 31, sub = lane & (L - 1), grp = lane / L;
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / L);
    double acc = 0.0;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L; r - grp < n; r += groups) {
        VT sum = r < n ? pad_row<VT, XT, L>(rp4, cp, vp, p, r, sub) : VT(0);
#pragma unroll
        for (int o = 1; o < L; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (sub == 0 && r < n) {
            q[r] = (XT)sum;
            acc += (double)p[r] * (double)sum;
        }
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0 && part) part[blockIdx.x] = t;
    if (st && last_block(st)) {
        const double pq = warp_sum_parts(part, gridDim.x);
        if (threadIdx.x == 0) {
            st->pq = pq;
            st->alpha = (pq != 0.0) ? st->rr / pq : 0.0;
            st->ticket = 0;
        }
    }
}

// r = b - A x (FP64) on the padded rows, with the partials of |r|^2
__global__ void __launch_bounds__(RB) k_residual_pad(const int64_t *__restrict__ rp4, const int32_t *__restrict__ cp,
                                                     const double *__restrict__ vp, const double *__restrict__ x,
                                                     const double *__restrict__ b, double *r, int64_t n, double *part)
{
    __shared__ double sh[RB / 32];
    const int lane = threadIdx.x & 31, sub = lane & 7, grp = lane >> 3;
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 3);
    double acc = 0.0;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3; row - grp < n; row += groups) {
        double sum = row < n ? pad_row<double, double>(rp4, cp, vp, x, row, sub) : 0.0;
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        sum += __shfl_xor_sync(0xffffffffu, sum, 4);
        if (sub == 0 && row < n) {
            const double ri = b[row] - sum;
            r[row] = ri;
            acc += ri * ri;
        }
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// With FUSE_P (small systems) the last block also updates p = r + beta p for
// every row (reading r and p through L2: other blocks wrote r), which saves
// the separate p launch of the iteration.
template <class XT, bool FUSE_P>
__global__ void k_update_xr(XT *x, XT *r, XT *p, const XT *q, int64_t n, double *part, CgState *st)
{
    __shared__ double sh[RB / 32];
    if (st->done) return;
    const XT a = (XT)st->alpha;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        XT ri = r[i] - a * q[i];
        r[i] = ri;
        acc += (double)ri * (double)ri;
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    // the last block forms beta = r'.r' / r.r and tests convergence
    if constexpr (!FUSE_P) {
        if (last_block(st)) {
            const double rr = warp_sum_parts(part, gridDim.x);
            if (threadIdx.x == 0) {
                st->beta = (st->rr != 0.0) ? rr / st->rr : 0.0;
                st->rr = rr;
                st->it += 1;
                if (rr <= st->tol2 || !(rr == rr)) st->done = 1;
                st->ticket = 0;
            }
        }
    } else {
        __shared__ bool last;
        __shared__ double beta_s;
        __shared__ int done_s;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
        __syncthreads();
        if (last) {                        // block-uniform
            if (threadIdx.x < 32) {
                const double rr = warp_sum_parts(part, gridDim.x);
                if (threadIdx.x == 0) {
                    const double beta = (st->rr != 0.0) ? rr / st->rr : 0.0;
                    const int done = (rr <= st->tol2 || !(rr == rr)) ? 1 : 0;
                    st->beta = beta;
                    st->rr = rr;
                    st->it += 1;
                    if (done) st->done = 1;
                    st->ticket = 0;
                    beta_s = beta;
                    done_s = done;
                }
            }
            __syncthreads();
            if (!done_s) {
                const XT b = (XT)beta_s;
                for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = __ldcg(r + i) + b * __ldcg(p + i);
            }
        }
    }
}

template <class XT>
__global__ void k_update_p(XT *p, const XT *r, int64_t n, const CgState *st)
{
    if (st->done) return;
    const XT b = (XT)st->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = r[i] + b * p[i];
}

template <class XT>
__global__ void k_init(const double *b, XT *x, XT *r, XT *p, int64_t n, double scale, double *part)
{
    __shared__ double sh[RB / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        XT v = (XT)(b[i] * scale);
        x[i] = XT(0);
        r[i] = v;
        p[i] = v;
        acc += (double)v * (double)v;
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_start(const double *part, int nb, double rtol2, CgState *st)
{
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];
    st->rr = s;
    st->tol2 = rtol2 * s;
    st->done = (s == 0.0) ? 1 : 0;
    st->it = 0;
    st->ticket = 0;
    st->alpha = st->beta = st->pq = 0.0;
    st->bar_count = 0;
    st->bar_gen = 0;
    st->bar_err = 0;
}

// Grid-wide barrier of a cooperative launch (all blocks resident).  The last
// block to arrive resets the count and advances the generation; the others
// wait for the new generation for at most wait_ns nanoseconds of the global
// timer (and at most 2^25 polls), then set the error flag and every block
// leaves: the host falls back to the multi-launch CG.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(CgState *st, unsigned long long wait_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = &st->bar_gen;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&st->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            st->bar_count = 0u;
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned int spins = 0;
            while (*gen == g) {
                if (++spins > (1u << 25) || global_ns() - t0 > wait_ns) {
                    atomicExch(&st->bar_err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok = *(volatile int *)&st->bar_err == 0;
    }
    __syncthreads();
    return ok != 0;
}

// Sum of the nb block partials in the fixed order of warp_sum_parts, formed by
// every block (the same value in all of them) and broadcast to its threads.
__device__ __forceinline__ double grid_sum(const double *part, int nb, double *bc)
{
    if (threadIdx.x < 32) {
        const double s = warp_sum_parts(part, nb);
        if (threadIdx.x == 0) *bc = s;
    }
    __syncthreads();
    const double v = *bc;
    __syncthreads();
    return v;
}

// The whole CG loop in one cooperative launch (small systems, where the
// launches of the multi-kernel loop dominate): per iteration q = A p with the
// partials of p.q, barrier, alpha, the x/r update with the partials of r.r,
// barrier, beta and the convergence test (the same in every block: the sums
// are formed in the same order), the p update, barrier.  Values another block
// wrote are read through L2.
template <class VT, class XT>
__global__ void __launch_bounds__(RB) k_cg_persist(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                   const VT *__restrict__ val, XT *x, XT *r, XT *p, XT *q, int64_t n,
                                                   double *part, double *part2, CgState *st, int max_it,
                                                   unsigned long long wait_ns)
{
    __shared__ double sh[RB / 32];
    __shared__ double bc;
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    double rr = st->rr;
    const double tol2 = st->tol2;
    int it = 0, done = 0;
    while (it < max_it) {
        double acc = 0.0;
        for (int64_t row = gt >> 5; row < n; row += warps) {
            VT sum = VT(0);
            for (int64_t e = rp[row] + lane; e < rp[row + 1]; e += 32) sum += val[e] * (VT)__ldcg(p + ci[e]);
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) {
                q[row] = (XT)sum;
                acc += (double)__ldcg(p + row) * (double)sum;
            }
        }
        double t = block_sum(acc, sh);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
        if (!grid_barrier(st, wait_ns)) break;
        const double pq = grid_sum(part, gridDim.x, &bc);
        const XT a = (XT)((pq != 0.0) ? rr / pq : 0.0);
        acc = 0.0;
        for (int64_t i = gt; i < n; i += gs) {
            x[i] += a * p[i];
            const XT ri = r[i] - a * __ldcg(q + i);
            r[i] = ri;
            acc += (double)ri * (double)ri;
        }
        t = block_sum(acc, sh);
        if (threadIdx.x == 0) part2[blockIdx.x] = t;
        if (!grid_barrier(st, wait_ns)) break;
        const double rn = grid_sum(part2, gridDim.x, &bc);
        const double beta = (rr != 0.0) ? rn / rr : 0.0;
        rr = rn;
        ++it;
        if (rn <= tol2 || !(rn == rn)) {
            done = 1;
            break;
        }
        const XT b = (XT)beta;
        for (int64_t i = gt; i < n; i += gs) p[i] = r[i] + b * p[i];
        if (!grid_barrier(st, wait_ns)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rr = rr;
        st->it = it;
        st->done = done;
    }
}

__global__ void k_add_scaled(double *x, const float *d, double scale, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += scale * (double)d[i];
}

__global__ void k_scatter_u(const double *x, const int32_t *free_nodes, const double *g, const uint8_t *node_free,
                            double *u, int64_t nv, int64_t nf)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv && !node_free[i]) u[i] = g[i];
    if (i < nf) u[free_nodes[i]] = x[i];
}

// Blocks of the CG's vector kernels and of the FP64 residual: up to 16
// blocks of 256 threads per SM and 32 threads per row, at most 4096 (the
// partials of the no-allocation solve).
int cg_blocks(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>((int64_t)nl_num_sms() * 16, 4096),
                                                       nl_cdiv<int64_t>(n * 32, RB)));
}

// Blocks of k_spmv_dot_pad: one row group per row up to the blocks resident
// at once (never more than cg_blocks, whose partials array the kernel
// writes).
template <class VT, class XT>
int spmv_blocks(int64_t n)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_dot_pad<VT, XT>, RB, 0) != cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        occ = 1;
    }
    const int64_t rows = nl_cdiv<int64_t>(n * spmv_lanes<VT>(), RB);
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>((int64_t)occ * nl_num_sms(), rows),
                                                       cg_blocks(n)));
}

// systems up to this many rows update p in the last block of the x/r update
// (one block then walks all rows: beyond a few thousand rows that serial tail
// costs more than the separate p launch)
constexpr int64_t kFuseRows = 8192;
// and up to this many run the whole loop in one cooperative launch (larger
// ones are bandwidth-bound and want more resident blocks than one per SM)
constexpr int64_t kPersistRows = 16384;

struct Cg {
    int fallbacks = 0;         // single-launch loops that gave up a barrier wait (redone with separate launches)
    int nb = 0;
    double *part = nullptr;
    double *part2 = nullptr;   // second partials of the single-launch CG (null: not used)
    CgState *st = nullptr;
};

// Longest wait of a grid barrier of the single-launch CG: one second, or the
// nanoseconds in NL_CG_BARRIER_WAIT_NS (a testing knob: 0 makes every wait
// give up at once, which exercises the multi-launch fallback).
unsigned long long barrier_wait_ns()
{
    const char *e = getenv("NL_CG_BARRIER_WAIT_NS");
    if (!e || !*e) return 1000000000ull;
    return strtoull(e, nullptr, 10);
}

// Blocks of the single-launch CG: all resident at once (a cooperative launch
// fails rather than oversubscribe), at most the partials' size.
template <class VT, class XT>
int persist_blocks(int nb)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_persist<VT, XT>, RB, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    // at most one block per SM: the iterations of these small systems are
    // latency-bound, and fewer blocks make the barriers cheaper
    return std::min(std::min(nb, occ * nl_num_sms()), nl_num_sms());
}

// Run CG from x = 0 on A x = b*scale; returns iterations; converged flag in *conv.
template <class VT, class XT>
int run_cg(const int64_t *rp, const int32_t *ci, const VT *val, const int64_t *rp4, const int32_t *cp, const VT *vp,
           const double *b, double scale, XT *x, XT *r, XT *p,
           XT *q, int64_t n, double rtol, int max_it, int check_every, Cg &cg, cudaStream_t s, bool *conv)
{
    const int nb = cg.nb;
    { k_init<XT><<<nb, RB, 0, s>>>(b, x, r, p, n, scale, cg.part); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    { k_start<<<1, 32, 0, s>>>(cg.part, nb, rtol * rtol, cg.st); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    CgState h{};
    int launched = 0;
    *conv = false;
    if (cg.part2 && n <= kPersistRows) {
        const int nbp = persist_blocks<VT, XT>(nb);
        if (nbp > 0) {
            unsigned long long wait_ns = barrier_wait_ns();
            void *args[] = {(void *)&rp, (void *)&ci, (void *)&val, (void *)&x, (void *)&r, (void *)&p, (void *)&q,
                            (void *)&n, (void *)&cg.part, (void *)&cg.part2, (void *)&cg.st, (void *)&max_it,
                            (void *)&wait_ns};
            const cudaError_t le = cudaLaunchCooperativeKernel((const void *)k_cg_persist<VT, XT>,
                                                               dim3((unsigned)nbp), dim3(RB), args, 0, s);
            if (le != cudaSuccess) (void)cudaGetLastError();     // not launched: the multi-launch loop below
            else nl_count_launch();
            NL_CUDA(cudaMemcpyAsync(&h, cg.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
            NL_CUDA(cudaStreamSynchronize(s));
            if (le == cudaSuccess && h.bar_err == 0) {
                *conv = h.done && (h.rr == h.rr);
                return h.it;
            }
            if (le == cudaSuccess) {
                // a barrier wait gave up: redo the solve with separate launches
                cg.fallbacks++;
                { k_init<XT><<<nb, RB, 0, s>>>(b, x, r, p, n, scale, cg.part); nl_count_launch(); }
                NL_CHECK_LAUNCH();
                { k_start<<<1, 32, 0, s>>>(cg.part, nb, rtol * rtol, cg.st); nl_count_launch(); }
                NL_CHECK_LAUNCH();
            }
        }
    }
    const int nbs = spmv_blocks<VT, XT>(n);
    while (launched < max_it) {
        int k = std::min(check_every, max_it - launched);
        for (int j = 0; j < k; ++j) {
            { k_spmv_dot_pad<VT, XT><<<nbs, RB, 0, s>>>(rp4, cp, vp, p, q, n, cg.part, cg.st); nl_count_launch(); }
            if (n <= kFuseRows) {
                { k_update_xr<XT, true><<<nb, RB, 0, s>>>(x, r, p, q, n, cg.part, cg.st); nl_count_launch(); }
            } else {
                { k_update_xr<XT, false><<<nb, RB, 0, s>>>(x, r, p, q, n, cg.part, cg.st); nl_count_launch(); }
                { k_update_p<XT><<<nb, RB, 0, s>>>(p, r, n, cg.st); nl_count_launch(); }
            }
        }
        NL_CHECK_LAUNCH();
        launched += k;
        NL_CUDA(cudaMemcpyAsync(&h, cg.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        if (h.done) break;
    }
    *conv = h.done && (h.rr == h.rr);
    return h.it;
}

}  // namespace

nl_status nl_solve_impl(nl_system *S, const nl_solve_opts *opts, double *u_out, int where, nl_solve_info *info)
{
    nl_pairs *P = S->pairs;
    nl_mesh *m = P->mesh;
    const int64_t n = m->n_free;
    double rtol = (opts && opts->rtol > 0) ? opts->rtol : 1e-12;
    int max_it = (opts && opts->max_iter > 0) ? opts->max_iter : 20000;
    int mixed = opts ? opts->mixed : 0;
    double inner = (opts && opts->inner_rtol > 0) ? opts->inner_rtol : 1e-5;
    int check_every = (opts && opts->check_every > 0) ? opts->check_every : 8;
    nl_solve_info inf{0, 0, 0.0, 0};
    nl_status ret = NL_OK;
    try {
        cudaStream_t s = S->arena.stream();
        Scratch sc(&S->arena);
        Cg cg;
        cg.nb = cg_blocks(n);
        cg.part = sc.get<double>(cg.nb);
        cg.part2 = sc.get<double>(cg.nb);
        cg.st = sc.get<CgState>(1);
        double *x = sc.get<double>(n);
        double *rres = sc.get<double>(n);
        // |b| (residual of u = 0)
        double bb = 0.0;
        {
            double *z = sc.get<double>(n);
            NL_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * n, s));
            { k_residual_pad<<<cg.nb, RB, 0, s>>>(P->ap_rowptr4, P->ap_col, S->Ap, z, S->b, rres, n, cg.part); nl_count_launch(); }
            NL_CHECK_LAUNCH();
            std::vector<double> hp(cg.nb);
            NL_CUDA(cudaMemcpyAsync(hp.data(), cg.part, sizeof(double) * cg.nb, cudaMemcpyDeviceToHost, s));
            NL_CUDA(cudaStreamSynchronize(s));
            for (double v : hp) bb += v;
        }
        const double nb_ = sqrt(bb);
        bool converged = false;
        if (!mixed) {
            double *r = sc.get<double>(n), *p = sc.get<double>(n), *q = sc.get<double>(n);
            bool conv = false;
            inf.iterations = run_cg<double, double>(P->a_rowptr, P->a_col, S->A, P->ap_rowptr4, P->ap_col, S->Ap, S->b, 1.0, x, r, p, q, n, rtol,
                                                    max_it, check_every, cg, s, &conv);
            converged = conv;
        } else {
            float *xf = sc.get<float>(n), *rf = sc.get<float>(n), *pf = sc.get<float>(n), *qf = sc.get<float>(n);
            NL_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
            int total = 0;
            for (int outer = 0; outer < 100 && total < max_it; ++outer) {
                { k_residual_pad<<<cg.nb, RB, 0, s>>>(P->ap_rowptr4, P->ap_col, S->Ap, x, S->b, rres, n, cg.part); nl_count_launch(); }
                NL_CHECK_LAUNCH();
                std::vector<double> hp(cg.nb);
                NL_CUDA(cudaMemcpyAsync(hp.data(), cg.part, sizeof(double) * cg.nb, cudaMemcpyDeviceToHost, s));
                NL_CUDA(cudaStreamSynchronize(s));
                double rr = 0.0;
                for (double v : hp) rr += v;
                if (sqrt(rr) <= rtol * nb_ || rr == 0.0) { converged = true; break; }
                double rn = sqrt(rr);
                bool conv = false;
                int it = run_cg<float, float>(P->a_rowptr, P->a_col, S->A32, P->ap_rowptr4, P->ap_col, S->Ap32, rres, 1.0 / rn, xf, rf, pf, qf, n,
                                              inner, max_it - total, check_every, cg, s, &conv);
                total += it;
                inf.refinements += 1;
                { k_add_scaled<<<cg.nb, RB, 0, s>>>(x, xf, rn, n); nl_count_launch(); }
                NL_CHECK_LAUNCH();
                if (it == 0) break;
            }
            inf.iterations = total;
        }
        // true residual
        { k_residual_pad<<<cg.nb, RB, 0, s>>>(P->ap_rowptr4, P->ap_col, S->Ap, x, S->b, rres, n, cg.part); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        std::vector<double> hp(cg.nb);
        NL_CUDA(cudaMemcpyAsync(hp.data(), cg.part, sizeof(double) * cg.nb, cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        double rr = 0.0;
        for (double v : hp) rr += v;
        inf.rel_residual = (nb_ > 0) ? sqrt(rr) / nb_ : 0.0;
        inf.barrier_fallbacks = cg.fallbacks;
        if (mixed) converged = inf.rel_residual <= rtol * 1.0000001;
        if (u_out) {
            double *u = (where == NL_DEVICE) ? u_out : sc.get<double>(m->nv);
            { k_scatter_u<<<(unsigned)nl_cdiv<int64_t>(std::max(m->nv, n), 256), 256, 0, s>>>(
                x, m->free_nodes, S->g, m->node_free, u, m->nv, n); nl_count_launch(); }
            NL_CHECK_LAUNCH();
            if (where == NL_HOST)
                NL_CUDA(cudaMemcpyAsync(u_out, u, sizeof(double) * m->nv, cudaMemcpyDeviceToHost, s));
            NL_CUDA(cudaStreamSynchronize(s));
        }
        if (!converged) {
            nl_set_error("CG stopped after %d iterations at relative residual %.3e", inf.iterations, inf.rel_residual);
            ret = NL_ENOTCONV;
        }
    } catch (NlError &e) {
        ret = e.st;
    }
    if (info) *info = inf;
    return ret;
}

namespace {
__global__ void k_fill_ones(double *a, float *b, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i] = 1.0; b[i] = 1.0f; }
}
}  // namespace

extern "C" nl_status nl_spmv_time(nl_system *S, int precision, int reps, int64_t flush_bytes, double *ms_per_spmv,
                                  double *bytes_per_spmv)
{
    nl_clear_error();
    if (!S || !ms_per_spmv || reps < 1 || flush_bytes < 0 || (precision != NL_FP64 && precision != NL_FP32_COMP)) {
        nl_set_error("bad argument");
        return NL_EINVAL;
    }
    try {
        const nl_pairs *P = S->pairs;
        const int64_t n = P->mesh->n_free, nnz = P->nnz_a;
        cudaStream_t s = S->arena.stream();
        Scratch sc(&S->arena);
        double *xd = sc.get<double>(n), *yd = sc.get<double>(n);
        float *xf = sc.get<float>(n), *yf = sc.get<float>(n);
        unsigned char *fl = flush_bytes > 0 ? sc.get<unsigned char>(flush_bytes) : nullptr;
        { k_fill_ones<<<(unsigned)nl_cdiv<int64_t>(n, 256), 256, 0, s>>>(xd, xf, n); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        const int nb = precision == NL_FP64 ? spmv_blocks<double, double>(n) : spmv_blocks<float, float>(n);
        auto launch = [&]() {
            if (precision == NL_FP64)
                { k_spmv_dot_pad<double, double><<<nb, RB, 0, s>>>(P->ap_rowptr4, P->ap_col, S->Ap, xd, yd, n, nullptr, nullptr); nl_count_launch(); }
            else
                { k_spmv_dot_pad<float, float><<<nb, RB, 0, s>>>(P->ap_rowptr4, P->ap_col, S->Ap32, xf, yf, n, nullptr, nullptr); nl_count_launch(); }
        };
        ScopedEvent e0, e1;
        launch();                                   // untimed
        float total = 0.f;
        if (!fl) {
            NL_CUDA(cudaEventRecord(e0, s));
            for (int k = 0; k < reps; ++k) launch();
            NL_CUDA(cudaEventRecord(e1, s));
            NL_CHECK_LAUNCH();
            NL_CUDA(cudaEventSynchronize(e1));
            NL_CUDA(cudaEventElapsedTime(&total, e0, e1));
        } else {
            // each launch alone after a write of flush_bytes (L2 holds none of A)
            for (int k = 0; k < reps; ++k) {
                NL_CUDA(cudaMemsetAsync(fl, k & 0xff, (size_t)flush_bytes, s));
                NL_CUDA(cudaEventRecord(e0, s));
                launch();
                NL_CUDA(cudaEventRecord(e1, s));
                NL_CHECK_LAUNCH();
                NL_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                NL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                total += ms;
            }
        }
        *ms_per_spmv = total / reps;
        const double vb = precision == NL_FP64 ? 8.0 : 4.0;
        if (bytes_per_spmv) *bytes_per_spmv = (double)nnz * (vb + 4.0) + (double)(n + 1) * 8.0 + 2.0 * n * vb;
    } catch (NlError &e) {
        return e.st;
    }
    return NL_OK;
}

extern "C" nl_status nl_solve(nl_system *S, const nl_solve_opts *opts, double *u_out, int where, nl_solve_info *info)
{
    nl_clear_error();
    if (!S) { nl_set_error("NULL system"); return NL_EINVAL; }
    if (u_out && where != NL_HOST && where != NL_DEVICE) { nl_set_error("bad where"); return NL_EINVAL; }
    return nl_solve_impl(S, opts, u_out, where, info);
}

// ===========================================================================
// nl_solve_static: the FP64 CG solve with its scratch vectors in a fixed
// device array compiled into the library, for callers that must not allocate
// device memory during the call.  The array is shared by every call in the
// process and keeps the last call's contents; each call overwrites what it
// reads before reading it.
namespace {

constexpr int64_t kStaticMaxFree = 131072;        // unknowns (free nodes)
constexpr int kStaticMaxBlocks = 4096;            // reduction partials
constexpr size_t kStaticVecBytes = sizeof(double) * (size_t)kStaticMaxFree;
constexpr size_t kStaticBytes = 5 * kStaticVecBytes + sizeof(double) * kStaticMaxBlocks + 256;
static_assert(sizeof(CgState) <= 256, "the CG state slot of the static array");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
static void *g_static_addr[kMaxDevices] = {nullptr};
static std::mutex g_static_mu;

// Device address of the array on the current device (looked up once per
// device, under a lock so that threads making their first call at once do not
// race; the host-side symbol is only a stand-in and is never dereferenced).
void *static_scratch_address()
{
    int dev = 0;
    NL_CUDA(cudaGetDevice(&dev));
    NL_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            nl_set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            throw NlError{NL_ECUDA};
        }
        g_static_addr[dev] = p;
    }
    return g_static_addr[dev];
}

// Whether ptr is device (or managed) memory that the current device can
// write: the kernels of the static solve write u_out directly.
bool is_device_pointer(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

extern "C" nl_status nl_solve_static(nl_system *S, const nl_solve_opts *opts, double *u_out, nl_solve_info *info)
{
    nl_clear_error();
    if (!S || !u_out) { nl_set_error("NULL system or output"); return NL_EINVAL; }
    nl_pairs *P = S->pairs;
    nl_mesh *m = P->mesh;
    const int64_t n = m->n_free;
    if (n > kStaticMaxFree) {
        nl_set_error("nl_solve_static supports at most %lld unknowns, the system has %lld",
                     (long long)kStaticMaxFree, (long long)n);
        return NL_EINVAL;
    }
    if (!is_device_pointer(u_out)) {
        nl_set_error("nl_solve_static: u_out must be device memory of the current device");
        return NL_EINVAL;
    }
    double rtol = (opts && opts->rtol > 0) ? opts->rtol : 1e-12;
    int max_it = (opts && opts->max_iter > 0) ? opts->max_iter : 20000;
    int check_every = (opts && opts->check_every > 0) ? opts->check_every : 8;
    nl_solve_info inf{0, 0, 0.0, 0};
    nl_status ret = NL_OK;
    try {
        cudaStream_t s = S->arena.stream();
        unsigned char *base = static_cast<unsigned char *>(static_scratch_address());
        double *x = reinterpret_cast<double *>(base);
        double *r = reinterpret_cast<double *>(base + 1 * kStaticVecBytes);
        double *p = reinterpret_cast<double *>(base + 2 * kStaticVecBytes);
        double *q = reinterpret_cast<double *>(base + 3 * kStaticVecBytes);
        double *rres = reinterpret_cast<double *>(base + 4 * kStaticVecBytes);
        Cg cg;
        cg.nb = cg_blocks(n);
        NL_REQUIRE(cg.nb <= kStaticMaxBlocks, "too many reduction blocks (%d)", cg.nb);
        cg.part = reinterpret_cast<double *>(base + 5 * kStaticVecBytes);
        cg.st = reinterpret_cast<CgState *>(base + 5 * kStaticVecBytes + sizeof(double) * kStaticMaxBlocks);
        double hp[kStaticMaxBlocks];
        // |b| from the residual of u = 0 (x starts at zero: clear it first)
        NL_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
        { k_residual_pad<<<cg.nb, RB, 0, s>>>(P->ap_rowptr4, P->ap_col, S->Ap, x, S->b, rres, n, cg.part); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        NL_CUDA(cudaMemcpyAsync(hp, cg.part, sizeof(double) * cg.nb, cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        double bb = 0.0;
        for (int i = 0; i < cg.nb; ++i) bb += hp[i];
        const double nb_ = sqrt(bb);
        bool conv = false;
        inf.iterations = run_cg<double, double>(P->a_rowptr, P->a_col, S->A, P->ap_rowptr4, P->ap_col, S->Ap, S->b, 1.0, x, r, p, q, n, rtol, max_it,
                                                check_every, cg, s, &conv);
        { k_residual_pad<<<cg.nb, RB, 0, s>>>(P->ap_rowptr4, P->ap_col, S->Ap, x, S->b, rres, n, cg.part); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        NL_CUDA(cudaMemcpyAsync(hp, cg.part, sizeof(double) * cg.nb, cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        double rr = 0.0;
        for (int i = 0; i < cg.nb; ++i) rr += hp[i];
        inf.rel_residual = (nb_ > 0) ? sqrt(rr) / nb_ : 0.0;
        inf.barrier_fallbacks = cg.fallbacks;
        { k_scatter_u<<<(unsigned)nl_cdiv<int64_t>(std::max(m->nv, n), 256), 256, 0, s>>>(
              x, m->free_nodes, S->g, m->node_free, u_out, m->nv, n); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        NL_CUDA(cudaStreamSynchronize(s));
        if (!conv) {
            nl_set_error("CG stopped after %d iterations at relative residual %.3e", inf.iterations, inf.rel_residual);
            ret = NL_ENOTCONV;
        }
    } catch (NlError &e) {
        ret = e.st;
    }
    if (info) *info = inf;
    return ret;
}
