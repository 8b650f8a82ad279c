// Diagnostic entry points: the device geometry and the Philox stream on
// caller-given cases (host arrays in, host arrays out; default stream,
// cudaMalloc'd temporaries).  Used by tests to compare single cases with the
// CPU reference; not on the assembly path.
#include "nl_internal.h"
#include "nl_quad.cuh"

void nl_probe_fp64(const double *, const double4 *, const double *, const uint32_t *, int64_t, double, int, int,
                   uint64_t, double *, int *);
void nl_probe_fp32(const double *, const double4 *, const double *, const uint32_t *, int64_t, double, int, int,
                   uint64_t, double *, int *);
void nl_probe_samples_fp64(const double *, const double4 *, const double *, const uint32_t *, int64_t, double, int,
                           uint64_t, int, double *, int *, double *, int *);
void nl_probe_samples_fp32(const double *, const double4 *, const double *, const uint32_t *, int64_t, double, int,
                           uint64_t, int, double *, int *, double *, int *);

namespace {
__global__ void k_philox(const uint4 *__restrict__ ctr, uint2 key, int64_t n, uint4 *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = nlq::philox4x32_10(ctr[i], key);
}

struct Tmp {
    std::vector<void *> p;
    template <class T> T *get(size_t n)
    {
        void *q = nullptr;
        NL_CUDA(cudaMalloc(&q, sizeof(T) * (n ? n : 1)));
        p.push_back(q);
        return (T *)q;
    }
    ~Tmp() { for (void *q : p) cudaFree(q); }
};
}  // namespace

extern "C" nl_status nl_probe_moments(const double *tets_xyz, const double *x, const uint32_t *ids, int64_t n,
                                      double delta, int strategy, int mc_points, uint64_t seed, int precision,
                                      double *moments)
{
    nl_clear_error();
    if (!tets_xyz || !x || !ids || !moments || n < 0) { nl_set_error("bad argument"); return NL_EINVAL; }
    if (strategy < 0 || strategy > NL_FULLCAPS_QMC || (precision != NL_FP64 && precision != NL_FP32_COMP)) {
        nl_set_error("bad strategy or precision");
        return NL_EINVAL;
    }
    if (n == 0) return NL_OK;
    try {
        Tmp t;
        double *dv = t.get<double>(12 * n), *dx = t.get<double>(3 * n), *dm = t.get<double>(15 * n);
        uint32_t *di = t.get<uint32_t>(3 * n);
        NL_CUDA(cudaMemcpy(dv, tets_xyz, sizeof(double) * 12 * n, cudaMemcpyHostToDevice));
        NL_CUDA(cudaMemcpy(dx, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
        NL_CUDA(cudaMemcpy(di, ids, sizeof(uint32_t) * 3 * n, cudaMemcpyHostToDevice));
        // the same coordinates as a vertex table (4 vertices per case) for the exact decisions
        std::vector<double4> h4(4 * n);
        for (int64_t i = 0; i < 4 * n; ++i)
            h4[i] = make_double4(tets_xyz[3 * i], tets_xyz[3 * i + 1], tets_xyz[3 * i + 2], 0.0);
        double4 *dv4 = t.get<double4>(4 * n);
        NL_CUDA(cudaMemcpy(dv4, h4.data(), sizeof(double4) * 4 * n, cudaMemcpyHostToDevice));
        int *dd = t.get<int>(n);
        if (precision == NL_FP64) nl_probe_fp64(dv, dv4, dx, di, n, delta * delta, strategy, mc_points, seed, dm, dd);
        else nl_probe_fp32(dv, dv4, dx, di, n, delta * delta, strategy, mc_points, seed, dm, dd);
        NL_CUDA(cudaMemcpy(moments, dm, sizeof(double) * 15 * n, cudaMemcpyDeviceToHost));
    } catch (NlError &e) {
        return e.st;
    }
    return NL_OK;
}

namespace {
nl_status probe_samples(const double *tets_xyz, const double *x, const uint32_t *ids, int64_t n, double delta,
                        int mc_points, uint64_t seed, int precision, int qmc, int32_t *n_samples, int32_t *cell,
                        uint8_t *accepted, double *y)
{
    nl_clear_error();
    if (!tets_xyz || !x || !ids || !n_samples || !cell || !accepted || !y || n < 0) {
        nl_set_error("bad argument");
        return NL_EINVAL;
    }
    if (mc_points < 1 || mc_points > 4096 || (precision != NL_FP64 && precision != NL_FP32_COMP)) {
        nl_set_error("mc_points outside 1..4096 or bad precision");
        return NL_EINVAL;
    }
    if (n == 0) return NL_OK;
    if (n > (int64_t)1 << 20) { nl_set_error("at most 2^20 cases per call"); return NL_EINVAL; }
    try {
        Tmp t;
        const int64_t ns = n * (int64_t)mc_points;
        double *dv = t.get<double>(12 * n), *dx = t.get<double>(3 * n), *dm = t.get<double>(15 * n);
        double *drec = t.get<double>(5 * ns);
        uint32_t *di = t.get<uint32_t>(3 * n);
        int *dd = t.get<int>(n), *dn = t.get<int>(n);
        NL_CUDA(cudaMemcpy(dv, tets_xyz, sizeof(double) * 12 * n, cudaMemcpyHostToDevice));
        NL_CUDA(cudaMemcpy(dx, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
        NL_CUDA(cudaMemcpy(di, ids, sizeof(uint32_t) * 3 * n, cudaMemcpyHostToDevice));
        std::vector<double4> h4(4 * n);
        for (int64_t i = 0; i < 4 * n; ++i)
            h4[i] = make_double4(tets_xyz[3 * i], tets_xyz[3 * i + 1], tets_xyz[3 * i + 2], 0.0);
        double4 *dv4 = t.get<double4>(4 * n);
        NL_CUDA(cudaMemcpy(dv4, h4.data(), sizeof(double4) * 4 * n, cudaMemcpyHostToDevice));
        NL_CUDA(cudaMemset(dn, 0, sizeof(int) * n));
        if (precision == NL_FP64)
            nl_probe_samples_fp64(dv, dv4, dx, di, n, delta * delta, mc_points, seed, qmc, dm, dd, drec, dn);
        else
            nl_probe_samples_fp32(dv, dv4, dx, di, n, delta * delta, mc_points, seed, qmc, dm, dd, drec, dn);
        std::vector<double> hrec(5 * ns);
        std::vector<int> hn(n);
        NL_CUDA(cudaMemcpy(hrec.data(), drec, sizeof(double) * 5 * ns, cudaMemcpyDeviceToHost));
        NL_CUDA(cudaMemcpy(hn.data(), dn, sizeof(int) * n, cudaMemcpyDeviceToHost));
        for (int64_t c = 0; c < n; ++c) {
            n_samples[c] = hn[c];
            for (int k = 0; k < mc_points; ++k) {
                const int64_t s = c * mc_points + k;
                const bool have = k < hn[c];
                const double *r = hrec.data() + 5 * s;
                cell[s] = have ? (int32_t)r[0] : -1;
                accepted[s] = have && r[1] != 0.0 ? 1 : 0;
                for (int d = 0; d < 3; ++d) {
                    // FP32 points are relative to the outer point
                    const double off = precision == NL_FP64 ? 0.0 : x[3 * c + d];
                    y[3 * s + d] = have ? (precision == NL_FP64 ? r[2 + d] : off + r[2 + d]) : 0.0;
                }
            }
        }
    } catch (NlError &e) {
        return e.st;
    }
    return NL_OK;
}
}  // namespace

extern "C" nl_status nl_probe_mc_samples(const double *tets_xyz, const double *x, const uint32_t *ids, int64_t n,
                                         double delta, int mc_points, uint64_t seed, int precision,
                                         int32_t *n_samples, int32_t *cell, uint8_t *accepted, double *y)
{
    return probe_samples(tets_xyz, x, ids, n, delta, mc_points, seed, precision, 0, n_samples, cell, accepted, y);
}

extern "C" nl_status nl_probe_qmc_samples(const double *tets_xyz, const double *x, const uint32_t *ids, int64_t n,
                                          double delta, int mc_points, uint64_t seed, int precision,
                                          int32_t *n_samples, int32_t *cell, uint8_t *accepted, double *y)
{
    return probe_samples(tets_xyz, x, ids, n, delta, mc_points, seed, precision, 1, n_samples, cell, accepted, y);
}

extern "C" nl_status nl_probe_philox(const uint32_t *ctr, uint64_t key, int64_t n, uint32_t *out)
{
    nl_clear_error();
    if (!ctr || !out || n < 0) { nl_set_error("bad argument"); return NL_EINVAL; }
    if (n == 0) return NL_OK;
    try {
        Tmp t;
        uint4 *dc = t.get<uint4>(n), *doo = t.get<uint4>(n);
        NL_CUDA(cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice));
        { k_philox<<<(unsigned)((n + 255) / 256), 256>>>(dc, make_uint2((uint32_t)key, (uint32_t)(key >> 32)), n, doo); nl_count_launch(); }
        NL_CHECK_LAUNCH();
        NL_CUDA(cudaMemcpy(out, doo, sizeof(uint4) * n, cudaMemcpyDeviceToHost));
    } catch (NlError &e) {
        return e.st;
    }
    return NL_OK;
}
