// FP64 assembly.  Compiled with -fmad=false: every decision of the method
// (inside test, edge/sphere points, diagonal, sampling volumes, Monte Carlo
// points and acceptance) follows the fixed operation order of the arithmetic
// specification, with no fused multiply-add.
#include "nl_assemble.cuh"

void nl_assemble_fp64(nl_system *sys, double *D, double *strips, double *TT, uint8_t *nfull, uint64_t *stats)
{
    nla::launch_assemble<double>(sys, D, strips, TT, nfull, reinterpret_cast<unsigned long long *>(stats));
}

void nl_probe_fp64(const double *tv, const double4 *tv4, const double *xs, const uint32_t *ids, int64_t n, double delta2, int strategy,
                   int nmc, uint64_t seed, double *out, int *defer)
{
    nla::launch_probe<double>(tv, tv4, xs, ids, n, delta2, strategy, nmc, seed, out, defer);
}

void nl_batch_alloc_work_fp64(nla::BatchGroup &g, DevArena &arena, int64_t max_units, std::vector<void *> &owned)
{
    nla::alloc_group_work<double>(g, arena, max_units, owned);
}

void nl_batch_launch_fp64(const nla::BatchGroup &g, const nla::Shape &sh, cudaStream_t s)
{
    nla::launch_group<double>(g, sh, s);
}

void nl_probe_samples_fp64(const double *tv, const double4 *tv4, const double *xs, const uint32_t *ids, int64_t n,
                          double delta2, int nmc, uint64_t seed, int qmc, double *out, int *defer, double *rec,
                          int *nrec)
{
    nla::launch_probe_samples<double>(tv, tv4, xs, ids, n, delta2, nmc, seed, qmc, out, defer, rec, nrec);
}
