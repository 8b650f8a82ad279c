// Error plumbing, device allocation through the caller's hooks, prefix sums
// and a segmented sort used when building pair lists and the sparsity pattern.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "nl_internal.h"

#include <atomic>

static thread_local char g_err[1024] = {0};
static std::atomic<unsigned long long> g_launches{0};

void nl_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void nl_count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void nl_uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
extern "C" uint64_t nl_kernel_launches(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

void nl_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void nl_clear_error() { g_err[0] = 0; }

extern "C" const char *nl_last_error(void) { return g_err; }
extern "C" const char *nl_version(void) { return "nlfem 0.1 (sm_103a)"; }

void *DevArena::raw(size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (dev.alloc) {
        p = dev.alloc(bytes, dev.ctx);
        if (!p) {
            nl_set_error("device allocation of %zu bytes failed", bytes);
            throw NlError{NL_ENOMEM};
        }
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            nl_set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
            throw NlError{e == cudaErrorMemoryAllocation ? NL_ENOMEM : NL_ECUDA};
        }
    }
    ptrs.push_back(p);
    return p;
}

void DevArena::release(void *p)
{
    if (!p) return;
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it == ptrs.end()) return;
    ptrs.erase(it);
    if (dev.free) {
        // stream-ordered callers (e.g. a caching allocator) may reuse the block
        // for later work on the same stream; other streams are not involved.
        dev.free(p, dev.ctx);
    } else {
        cudaStreamSynchronize(stream());
        cudaFree(p);
    }
}

void DevArena::release_all()
{
    if (!ptrs.empty() && !dev.free) cudaStreamSynchronize(stream());
    for (size_t i = ptrs.size(); i-- > 0;) {
        if (dev.free) dev.free(ptrs[i], dev.ctx);
        else cudaFree(ptrs[i]);
    }
    ptrs.clear();
}

int nl_num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------------------
// exclusive scan of int64 (three phases, recursive on the block sums)
static constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v)
{
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += t;
    }
    return v;
}

__global__ void k_scan_block(const int64_t *in, int64_t *out, int64_t *bsum, int64_t n)
{
    __shared__ int64_t ws[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int64_t v = (i < n) ? in[i] : 0;
    int64_t inc = warp_incl_scan(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t t = ws[lane];
        t = warp_incl_scan(t);
        ws[lane] = t;
    }
    __syncthreads();
    int64_t base = (w > 0) ? ws[w - 1] : 0;
    if (i < n) out[i] = base + inc - v;
    if (threadIdx.x == SCAN_BLOCK - 1) bsum[blockIdx.x] = base + inc;
}

__global__ void k_scan_add(int64_t *out, const int64_t *boff, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

void nl_exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, DevArena *arena, cudaStream_t s)
{
    if (n <= 0) return;
    int64_t nb = nl_cdiv<int64_t>(n, SCAN_BLOCK);
    Scratch sc(arena);
    int64_t *bsum = sc.get<int64_t>(nb);
    { k_scan_block<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, out, bsum, n); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    if (nb > 1) {
        int64_t *boff = sc.get<int64_t>(nb);
        nl_exclusive_scan_i64(bsum, boff, nb, arena, s);
        { k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(out, boff, n); nl_count_launch(); }
        NL_CHECK_LAUNCH();
    }
}

__global__ void k_set_last(int64_t *out, const int64_t *counts, int64_t n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) out[n] = (n > 0 ? out[n - 1] + counts[n - 1] : 0);
}

int64_t nl_scan_counts(const int64_t *counts, int64_t *out, int64_t n, DevArena *arena, cudaStream_t s)
{
    nl_exclusive_scan_i64(counts, out, n, arena, s);
    { k_set_last<<<1, 32, 0, s>>>(out, counts, n); nl_count_launch(); }
    NL_CHECK_LAUNCH();
    int64_t total = 0;
    NL_CUDA(cudaMemcpyAsync(&total, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NL_CUDA(cudaStreamSynchronize(s));
    return total;
}

// ---------------------------------------------------------------------------
// segmented sort: one block per segment, bitonic sort in shared memory
__global__ void k_seg_bitonic(int32_t *keys, const int64_t *ptr, int pow2)
{
    extern __shared__ int32_t sk[];
    int64_t b = ptr[blockIdx.x], e = ptr[blockIdx.x + 1];
    int n = (int)(e - b);
    if (n <= 1) return;
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) sk[i] = (i < n) ? keys[b + i] : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    int32_t a = sk[i], c = sk[ixj];
                    bool up = ((i & k) == 0);
                    if ((a > c) == up) { sk[i] = c; sk[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) keys[b + i] = sk[i];
    (void)pow2;
}

// Segments of up to 1024 keys: one warp per segment, K keys per lane in
// registers (key i = 32 r + lane in register r), the same bitonic network:
// partners 32 or more apart are in the same lane (register exchange), closer
// ones in another lane (shuffle).  No block barrier.
template <int K>
__device__ __forceinline__ void warp_bitonic(int32_t *keys, int64_t b, int n, int lane)
{
    int32_t v[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int i = 32 * r + lane;
        v[r] = i < n ? keys[b + i] : 0x7fffffff;
    }
    constexpr int P = 32 * K;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int rj = j >> 5;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    if ((r & rj) == 0) {
                        const bool up = ((32 * r + lane) & k) == 0;
                        const int32_t a = v[r], c = v[r | rj];
                        const int32_t lo = a < c ? a : c, hi = a < c ? c : a;
                        v[r] = up ? lo : hi;
                        v[r | rj] = up ? hi : lo;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const int i = 32 * r + lane;
                    const int32_t w = __shfl_xor_sync(0xffffffffu, v[r], j);
                    const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
                    v[r] = keep_min ? (v[r] < w ? v[r] : w) : (v[r] < w ? w : v[r]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int i = 32 * r + lane;
        if (i < n) keys[b + i] = v[r];
    }
}

__global__ void k_seg_warp(int32_t *keys, const int64_t *ptr, int64_t nseg)
{
    const int64_t sg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sg >= nseg) return;                 // warp-uniform
    const int64_t b = ptr[sg];
    const int n = (int)(ptr[sg + 1] - b);
    if (n <= 1) return;
    if (n <= 32) warp_bitonic<1>(keys, b, n, lane);
    else if (n <= 64) warp_bitonic<2>(keys, b, n, lane);
    else if (n <= 128) warp_bitonic<4>(keys, b, n, lane);
    else if (n <= 256) warp_bitonic<8>(keys, b, n, lane);
    else if (n <= 512) warp_bitonic<16>(keys, b, n, lane);
    else warp_bitonic<32>(keys, b, n, lane);
}

// Segments of 1025..2048 keys: two warps per segment, each sorting one half
// of up to 1024 keys in registers (warp_bitonic<32>, in place), then a merge
// through shared memory: every key of one half finds its rank in the other
// by binary search (lower bound for the first half, upper bound for the
// second, so that equal keys keep the order of the halves) and goes to its
// own index plus that rank.  Shorter segments in the same launch take the
// one-warp path.
__global__ void __launch_bounds__(64) k_seg_2k(int32_t *keys, const int64_t *ptr, int64_t nseg)
{
    __shared__ int32_t sh[2048];
    const int64_t sg = blockIdx.x;
    if (sg >= nseg) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t b = ptr[sg];
    const int n = (int)(ptr[sg + 1] - b);
    if (n <= 1024) {
        if (w == 0 && n > 1) {
            if (n <= 512) warp_bitonic<16>(keys, b, n, lane);
            else warp_bitonic<32>(keys, b, n, lane);
        }
        return;
    }
    const int na = 1024, nb = n - 1024;      // n <= 2048
    if (w == 0) warp_bitonic<32>(keys, b, na, lane);
    else warp_bitonic<32>(keys, b + na, nb, lane);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += 64) sh[i] = keys[b + i];
    __syncthreads();
    const int32_t *A = sh, *Bv = sh + na;
    for (int i = threadIdx.x; i < n; i += 64) {
        const int32_t k = sh[i];
        int lo = 0, hi;
        if (i < na) {
            hi = nb;                          // lower bound of k in B
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (Bv[mid] < k) lo = mid + 1; else hi = mid; }
            keys[b + i + lo] = k;
        } else {
            hi = na;                          // upper bound of k in A
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (A[mid] <= k) lo = mid + 1; else hi = mid; }
            keys[b + (i - na) + lo] = k;
        }
    }
}

void nl_segmented_sort_i32(int32_t *keys, const int64_t *ptr, int64_t nseg, int64_t max_seg,
                           DevArena *arena, cudaStream_t s)
{
    (void)arena;
    if (nseg <= 0 || max_seg <= 1) return;
    if (max_seg <= 1024) {
        const int64_t blocks = (nseg + 7) / 8;     // 8 warps (segments) per block
        for (int64_t b0 = 0; b0 < blocks; b0 += 2147483647LL) {
            const int64_t nb = std::min<int64_t>(blocks - b0, 2147483647LL);
            { k_seg_warp<<<(unsigned)nb, 256, 0, s>>>(keys, ptr + 8 * b0, nseg - 8 * b0); nl_count_launch(); }
            NL_CHECK_LAUNCH();
        }
        return;
    }
    if (max_seg <= 2048) {
        for (int64_t s0 = 0; s0 < nseg; s0 += 2147483647LL) {
            const int64_t cnt = std::min<int64_t>(nseg - s0, 2147483647LL);
            { k_seg_2k<<<(unsigned)cnt, 64, 0, s>>>(keys, ptr + s0, cnt); nl_count_launch(); }
            NL_CHECK_LAUNCH();
        }
        return;
    }
    NL_REQUIRE(max_seg <= 32768, "a segment of %lld entries exceeds the 32768 supported by the sort",
               (long long)max_seg);
    int p2 = 1;
    while (p2 < max_seg) p2 <<= 1;
    // 128-thread blocks: most segments are far shorter than the longest, and
    // small blocks keep more segments in flight per SM
    int threads = std::min(128, std::max(32, p2 / 2));
    size_t smem = sizeof(int32_t) * (size_t)p2;
    // one process-wide limit for every size (concurrent callers never lower it)
    if (smem > 48 * 1024)
        NL_CUDA(cudaFuncSetAttribute(k_seg_bitonic, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(int32_t) * 32768)));
    for (int64_t s0 = 0; s0 < nseg; s0 += 2147483647LL) {
        int64_t cnt = std::min<int64_t>(nseg - s0, 2147483647LL);
        { k_seg_bitonic<<<(unsigned)cnt, threads, smem, s>>>(keys, ptr + s0, p2); nl_count_launch(); }
        NL_CHECK_LAUNCH();
    }
}
