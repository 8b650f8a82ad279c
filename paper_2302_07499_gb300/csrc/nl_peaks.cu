// Measured ALU rates of this GPU: the denominators of the assembly kernels'
// ALU roofline.  Each microbenchmark runs independent dependency chains in
// registers only (no memory traffic inside the timed loop) on a grid of
// resident blocks, and is timed with CUDA events:
//   0 FP32 FFMA           one fused multiply-add = 1 op
//   1 FP64 DFMA           1 op
//   2 INT32 mad.lo        1 op (the Philox multiply's low word)
//   3 INT32 mul.hi        1 op (the Philox multiply's high word)
//   4 3-input xor (lop3)  2 ops (two binary xors)
//   5 Philox4x32-10       80 ops per draw (10 rounds x (2 mul.lo + 2 mul.hi + 4 xor))
//   6 the fullcaps sample 121 ops per sample: a Philox draw (80), the cell
//                          choice (6), three uniforms (9), their sort (6), the
//                          spacings (4), the point (12), the ball test (4) --
//                          the per-sample count of the method's arithmetic,
//                          on cells held in registers
// Chains use inline PTX so that the compiler can neither fold nor
// reassociate them.  The result is stored only under a condition the
// compiler cannot decide, so no chain is dead.
#include "nl_asm_types.h"
#include "nl_internal.h"
#include "nl_quad.cuh"

namespace {

struct PkKeys {
    uint32_t k[20];
};

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) k_pk_ffma(int iters, float b, float c, float *sink)
{
    float a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(b), "f"(c));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_pk_dfma(int iters, double b, double c, double *sink)
{
    double a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(b), "d"(c));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
    if (s == 1234.5) sink[threadIdx.x] = s;
}

// kind 0: mad.lo.u32 a = a*m + c; 1: mul.hi.u32 a = hi(a*m); 2: lop3 a = a ^ m ^ c
template <int KIND>
__global__ void __launch_bounds__(PK_THREADS) k_pk_int(int iters, uint32_t m, uint32_t c, uint32_t *sink)
{
    uint32_t a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = threadIdx.x * 2654435761u + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) {
                if constexpr (KIND == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(m), "r"(c));
                else if constexpr (KIND == 1) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(m));
                else asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(m), "r"(c));
            }
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s ^= a[k];
    if (s == 0x9E3779B9u) sink[threadIdx.x] = s;
}

// Philox4x32-10 draws: 4 independent counters per thread.
__global__ void __launch_bounds__(PK_THREADS) k_pk_philox(int iters, const __grid_constant__ PkKeys K, uint32_t *sink)
{
    const uint32_t *rk = K.k;
    uint32_t s = 0;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint4 u = nlq::philox_rk(make_uint4(t, (uint32_t)i, (uint32_t)k, 7u), rk);
            s ^= (u.x ^ u.y) ^ (u.z ^ u.w);
        }
    }
    if (s == 0x9E3779B9u) sink[threadIdx.x] = s;
}

// The fullcaps sample's arithmetic on a cap cell held in registers: the
// Philox draw, the cell choice against two thresholds (kept in the result),
// three FP32 uniforms, their sort, the spacings, the point and the ball test.
__global__ void __launch_bounds__(PK_THREADS) k_pk_sample(int iters, const __grid_constant__ PkKeys K, float d2,
                                                          uint32_t *sink)
{
    const uint32_t *rk = K.k;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float c[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) c[k] = 0.01f * (float)((t + 3 * k) & 63) - 0.3f;
    const uint32_t t0 = 0x55555555u + (t & 255), t1 = 0xAAAAAAAAu - (t & 255);
    uint32_t acc = 0;
    for (int i = 0; i < iters; ++i) {
        const uint4 u = nlq::philox_rk(make_uint4(t, (uint32_t)i, 3u, 5u), rk);
        const uint32_t j = (u.x > t0 ? 1u : 0u) + (u.x > t1 ? 1u : 0u);
        const float U0 = nlq::unif<float>(u.y), U1 = nlq::unif<float>(u.z), U2 = nlq::unif<float>(u.w);
        const float lo = fminf(U0, U1), hi = fmaxf(U0, U1);
        const float s0 = fminf(lo, U2), mid = fmaxf(lo, U2);
        const float s1 = fminf(hi, mid), s2 = fmaxf(hi, mid);
        const float b0 = s0, b1 = s1 - s0, b2 = s2 - s1;
        const float wx = ((c[0] + b0 * c[3]) + b1 * c[6]) + b2 * c[9];
        const float wy = ((c[1] + b0 * c[4]) + b1 * c[7]) + b2 * c[10];
        const float wz = ((c[2] + b0 * c[5]) + b1 * c[8]) + b2 * c[11];
        acc += (((wx * wx + wy * wy) + wz * wz) <= d2 ? 1u : 0u) + j;
    }
    if (acc == 0x9E3779B9u) sink[threadIdx.x] = acc;
}

}  // namespace

extern "C" nl_status nl_probe_alu_rates(double *ops_per_s, int n)
{
    nl_clear_error();
    if (!ops_per_s || n < 7) { nl_set_error("ops_per_s needs 7 entries"); return NL_EINVAL; }
    try {
        int dev = 0, sms = 0;
        NL_CUDA(cudaGetDevice(&dev));
        NL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        void *sink = nullptr;
        NL_CUDA(cudaMalloc(&sink, sizeof(double) * PK_THREADS));
        cudaEvent_t e0, e1;
        NL_CUDA(cudaEventCreate(&e0));
        NL_CUDA(cudaEventCreate(&e1));
        PkKeys K;
        nla::philox_round_keys(0x0123456789ABCDEFull, K.k);
        // 8 blocks of 256 threads per SM: 64 resident warps, every scheduler full
        const unsigned blocks = (unsigned)(8 * sms);
        const double threads = (double)blocks * PK_THREADS;
        auto run = [&](int which, int iters) {
            switch (which) {
            case 0: k_pk_ffma<<<blocks, PK_THREADS>>>(iters, 0.999999f, 1e-7f, (float *)sink); break;
            case 1: k_pk_dfma<<<blocks, PK_THREADS>>>(iters, 0.999999, 1e-7, (double *)sink); break;
            case 2: k_pk_int<0><<<blocks, PK_THREADS>>>(iters, 0xD2511F53u, 0x9E3779B9u, (uint32_t *)sink); break;
            case 3: k_pk_int<1><<<blocks, PK_THREADS>>>(iters, 0xCD9E8D57u, 0u, (uint32_t *)sink); break;
            case 4: k_pk_int<2><<<blocks, PK_THREADS>>>(iters, 0xD2511F53u, 0x9E3779B9u, (uint32_t *)sink); break;
            case 5: k_pk_philox<<<blocks, PK_THREADS>>>(iters, K, (uint32_t *)sink); break;
            default: k_pk_sample<<<blocks, PK_THREADS>>>(iters, K, 0.05f, (uint32_t *)sink); break;
            }
            nl_count_launch();
        };
        // operations per thread and iteration
        const double per_iter[7] = {16.0 * PK_CHAINS, 16.0 * PK_CHAINS, 16.0 * PK_CHAINS, 16.0 * PK_CHAINS,
                                    2.0 * 16 * PK_CHAINS, 4.0 * 80, 121.0};
        const int iters[7] = {2048, 64, 1024, 1024, 1024, 512, 2048};
        for (int w = 0; w < 7; ++w) {
            run(w, iters[w] / 8);      // warm-up
            NL_CHECK_LAUNCH();
            float best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                NL_CUDA(cudaEventRecord(e0));
                run(w, iters[w]);
                NL_CUDA(cudaEventRecord(e1));
                NL_CUDA(cudaEventSynchronize(e1));
                NL_CHECK_LAUNCH();
                float ms = 0.f;
                NL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                best = ms < best ? ms : best;
            }
            ops_per_s[w] = threads * iters[w] * per_iter[w] / (best * 1e-3);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(sink);
    } catch (NlError &e) {
        return e.st;
    }
    return NL_OK;
}
