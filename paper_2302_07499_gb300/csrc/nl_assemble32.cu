// FP32 assembly: per-(pair, point) geometry, Monte Carlo and moments in FP32
// on coordinates relative to the outer point; every sum across points,
// pairs and elements is accumulated in FP64 (strips, staged moments, V_q).
#include "nl_assemble.cuh"

void nl_assemble_fp32(nl_system *sys, float *D, double *strips, double *TT, uint8_t *nfull, uint64_t *stats)
{
    nla::launch_assemble<float>(sys, D, strips, TT, nfull, reinterpret_cast<unsigned long long *>(stats));
}

void nl_probe_fp32(const double *tv, const double4 *tv4, const double *xs, const uint32_t *ids, int64_t n, double delta2, int strategy,
                   int nmc, uint64_t seed, double *out, int *defer)
{
    nla::launch_probe<float>(tv, tv4, xs, ids, n, delta2, strategy, nmc, seed, out, defer);
}

void nl_batch_alloc_work_fp32(nla::BatchGroup &g, DevArena &arena, int64_t max_units, std::vector<void *> &owned)
{
    nla::alloc_group_work<float>(g, arena, max_units, owned);
}

void nl_batch_launch_fp32(const nla::BatchGroup &g, const nla::Shape &sh, cudaStream_t s)
{
    nla::launch_group<float>(g, sh, s);
}

void nl_probe_samples_fp32(const double *tv, const double4 *tv4, const double *xs, const uint32_t *ids, int64_t n,
                          double delta2, int nmc, uint64_t seed, int qmc, double *out, int *defer, double *rec,
                          int *nrec)
{
    nla::launch_probe_samples<float>(tv, tv4, xs, ids, n, delta2, nmc, seed, qmc, out, defer, rec, nrec);
}
