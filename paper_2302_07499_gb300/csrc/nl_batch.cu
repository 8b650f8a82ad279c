// Batched assembly: many independent problems (each with its own mesh,
// pairs, delta and options) assembled by shared launches.
//
// The problems are grouped by (precision, strategy, Monte Carlo count, seed).
// Each group runs the three quadrature kernels once per chunk over the
// concatenated pair index space of its problems; every pair finds its problem
// through a pair -> problem map.  The arithmetic of every (pair, point) unit
// and the order of every sum are those of the problem alone, so a problem's K,
// A and b are bitwise equal to its single-problem assembly.  The reductions
// into CSR follow per problem.
//
// The autotuner times candidate launch shapes (chunk size, classification
// block size, resident event blocks per SM) on the batch itself and keeps the
// fastest.  The whole launch sequence is then captured once in a CUDA graph
// and replayed by nl_batch_run.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "nl_asm_types.h"
#include "nl_internal.h"

namespace {

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

struct nl_batch {
    DevArena arena;                       // batch-owned device memory
    std::vector<void *> owned;
    std::vector<nl_system *> sys;         // one per problem, in the caller's order
    std::vector<void *> D;                // per problem: staged T'T' moments
    std::vector<double *> strips, TT, G, E;
    std::vector<uint8_t *> nfull;         // FP32 problems: per pair, the points at which T' is whole
    std::vector<nla::BatchGroup> groups;
    unsigned long long *stats = nullptr;  // [8] summed over the batch
    nla::Shape shape;
    bool use_graph = false;
    cudaStream_t bs = nullptr;            // the batch's own stream (capturable), joined to the caller's
    cudaEvent_t join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches_per_run = 0;
    double last_ms = 0.0;
    int n_tried = 0;
    nla::Shape tried[16];
    double tried_ms[16];
};

namespace {

void batch_free(nl_batch *b)
{
    if (!b) return;
    if (b->bs) cudaStreamSynchronize(b->bs);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->join) cudaEventDestroy(b->join);
    if (b->bs) cudaStreamDestroy(b->bs);
    for (nl_system *s : b->sys) nl_system_destroy(s);
    b->arena.release_all();
    delete b;
}

// Every launch of one batch run, stream-ordered, without synchronisation.
void batch_enqueue(nl_batch *b, const nla::Shape &sh, cudaStream_t s)
{
    NL_CUDA(cudaMemsetAsync(b->stats, 0, 8 * sizeof(unsigned long long), s));
    for (auto &g : b->groups) {
        if (g.precision == NL_FP32_COMP) nl_batch_launch_fp32(g, sh, s);
        else nl_batch_launch_fp64(g, sh, s);
    }
    for (size_t i = 0; i < b->sys.size(); ++i) {
        nl_system *S = b->sys[i];
        nl_reduce_system_into(S, b->D[i], S->opts.precision == NL_FP32_COMP ? 1 : 0, b->nfull[i], b->strips[i],
                              b->TT[i], b->G[i], b->E[i], s);
    }
}

// One timed run of the batch with the given shape (ms).
double batch_time(nl_batch *b, const nla::Shape &sh, cudaStream_t s)
{
    ScopedEvent e0, e1;
    NL_CUDA(cudaEventRecord(e0, s));
    batch_enqueue(b, sh, s);
    NL_CUDA(cudaEventRecord(e1, s));
    NL_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    NL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
}

}  // namespace

extern "C" nl_status nl_batch_create(nl_pairs *const *pairs, const nl_assemble_opts *opts, int n,
                                     const nl_batch_opts *bopts, nl_batch **out)
{
    nl_clear_error();
    if (!pairs || !opts || !out || n < 1) { nl_set_error("bad argument"); return NL_EINVAL; }
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!pairs[i]) { nl_set_error("pairs[%d] is NULL", i); return NL_EINVAL; }
        if (nl_status st = nl_check_assemble_opts(&opts[i])) return st;
        if (opts[i].kernel_poly) { nl_set_error("a kernel shape (kernel_poly) runs through nl_assemble only"); return NL_EINVAL; }
        if (pairs[i]->arena.dev.stream != pairs[0]->arena.dev.stream) {
            nl_set_error("all problems of a batch must use the same stream");
            return NL_EINVAL;
        }
    }
    nl_batch *b = new nl_batch();
    b->arena.dev = pairs[0]->arena.dev;
    b->use_graph = bopts ? bopts->use_graph != 0 : true;
    const bool autotune = bopts ? bopts->autotune != 0 : true;
    try {
        cudaStream_t s = b->arena.stream();
        auto own = [&](void *p) { b->owned.push_back(p); return p; };
        b->stats = (unsigned long long *)own(b->arena.get<unsigned long long>(8));
        // per-problem systems and outputs
        for (int i = 0; i < n; ++i) {
            nl_pairs *P = pairs[i];
            nl_mesh *m = P->mesh;
            nl_system *S = nl_system_alloc(P, &opts[i]);
            b->sys.push_back(S);
            S->stats.pairs = (uint64_t)P->npairs;
            const bool f32 = opts[i].precision == NL_FP32_COMP;
            b->D.push_back(own(f32 ? (void *)b->arena.get<float>(10 * P->npairs)
                                   : (void *)b->arena.get<double>(10 * P->npairs)));
            b->strips.push_back((double *)own(b->arena.get<double>(P->strip_total)));
            b->TT.push_back((double *)own(b->arena.get<double>(10 * m->n_outer)));
            b->G.push_back((double *)own(b->arena.get<double>(P->nnz)));
            b->E.push_back((double *)own(b->arena.get<double>(10 * m->nt)));
            b->nfull.push_back(f32 ? (uint8_t *)own(b->arena.get<uint8_t>(P->npairs)) : nullptr);
        }
        // groups
        std::map<std::tuple<int, int, int, uint64_t>, std::vector<int>> gm;
        for (int i = 0; i < n; ++i) {
            const int nmc = (opts[i].strategy == NL_FULLCAPS || opts[i].strategy == NL_FULLCAPS_QMC)
                                ? opts[i].mc_points : 0;
            gm[std::make_tuple(opts[i].precision, opts[i].strategy, nmc, opts[i].seed)].push_back(i);
        }
        std::vector<std::vector<int64_t>> hptr(n);
        for (int i = 0; i < n; ++i) {
            nl_mesh *m = pairs[i]->mesh;
            hptr[i].resize(m->n_outer + 1);
            NL_CUDA(cudaMemcpyAsync(hptr[i].data(), pairs[i]->pair_ptr, sizeof(int64_t) * (m->n_outer + 1),
                                    cudaMemcpyDeviceToHost, s));
        }
        NL_CUDA(cudaStreamSynchronize(s));
        for (auto &kv : gm) {
            nla::BatchGroup g;
            memset(&g.A, 0, sizeof(g.A));
            const std::vector<int> &ids = kv.second;
            const nl_assemble_opts &o0 = opts[ids[0]];
            g.precision = o0.precision;
            g.strategy = o0.strategy;
            int max_row = 0;
            int64_t np_tot = 0, no_tot = 0;
            std::vector<nla::Prob> probs;
            for (int i : ids) {
                nla::Prob pr = nla::make_prob(b->sys[i], b->D[i], b->strips[i], b->TT[i], b->nfull[i]);
                pr.pair_base = np_tot;
                pr.outer_base = no_tot;
                probs.push_back(pr);
                max_row = std::max<int>(max_row, pairs[i]->max_row);
                // running pair count over the group's outer elements
                const std::vector<int64_t> &hp = hptr[i];
                if (g.gptr.empty()) g.gptr.push_back(0);
                for (size_t k = 1; k < hp.size(); ++k) g.gptr.push_back(np_tot + hp[k]);
                np_tot += pairs[i]->npairs;
                no_tot += pairs[i]->mesh->n_outer;
            }
            NL_REQUIRE(np_tot < 0x7fffffffLL, "a batch group of %lld pairs exceeds the int32 index", (long long)np_tot);
            nla::Prob *dprobs = (nla::Prob *)own(b->arena.get<nla::Prob>(probs.size()));
            NL_CUDA(cudaMemcpyAsync(dprobs, probs.data(), sizeof(nla::Prob) * probs.size(), cudaMemcpyHostToDevice, s));
            int32_t *pair_prob = (int32_t *)own(b->arena.get<int32_t>(np_tot));
            int32_t *outer_prob = (int32_t *)own(b->arena.get<int32_t>(no_tot));
            for (size_t k = 0; k < ids.size(); ++k) {
                const int64_t np = pairs[ids[k]]->npairs, no = pairs[ids[k]]->mesh->n_outer;
                if (np > 0) {
                    k_fill_i32<<<(unsigned)nl_cdiv<int64_t>(np, 256), 256, 0, s>>>(pair_prob + probs[k].pair_base, np,
                                                                                 (int32_t)k);
                    nl_count_launch();
                    NL_CHECK_LAUNCH();
                }
                if (no > 0) {
                    k_fill_i32<<<(unsigned)nl_cdiv<int64_t>(no, 256), 256, 0, s>>>(outer_prob + probs[k].outer_base, no,
                                                                                 (int32_t)k);
                    nl_count_launch();
                    NL_CHECK_LAUNCH();
                }
            }
            nla::init_group_args(g.A, o0, b->stats, max_row);
            g.A.probs = dprobs;
            g.A.pair_prob = pair_prob;
            g.A.outer_prob = outer_prob;
            b->groups.push_back(std::move(g));
        }
        // the batch runs on its own stream, which a graph can be captured on
        // (the caller's stream may be the legacy default stream)
        NL_CUDA(cudaStreamSynchronize(s));
        NL_CUDA(cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking));
        NL_CUDA(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
        // candidate shapes, and work arrays for the largest chunk any of them forms
        std::vector<nla::Shape> cands;
        const int64_t units[3] = {int64_t(1) << 23, int64_t(1) << 24, int64_t(1) << 25};
        const int cthreads[2] = {128, 256};
        if (autotune) {
            for (int64_t u : units)
                for (int ct : cthreads) {
                    nla::Shape sh;
                    sh.units_per_chunk = u;
                    sh.classify_threads = ct;
                    cands.push_back(sh);
                }
        } else {
            nla::Shape sh;
            if (bopts && bopts->units_per_chunk > 0) sh.units_per_chunk = bopts->units_per_chunk;
            if (bopts && bopts->classify_threads > 0) sh.classify_threads = bopts->classify_threads;
            NL_REQUIRE(sh.units_per_chunk >= 4096 && sh.units_per_chunk <= (int64_t(1) << 28) &&
                           (sh.classify_threads == 128 || sh.classify_threads == 256),
                       "bad launch shape (units per chunk %lld, classification block %d)",
                       (long long)sh.units_per_chunk, sh.classify_threads);
            cands.push_back(sh);
        }
        for (auto &g : b->groups) {
            int64_t mu = 0;
            for (auto &sh : cands) {
                int64_t m1 = 0;
                nla::plan_chunks(g.gptr, sh.units_per_chunk, &m1);
                mu = std::max(mu, m1);
            }
            if (g.precision == NL_FP32_COMP) nl_batch_alloc_work_fp32(g, b->arena, mu, b->owned);
            else nl_batch_alloc_work_fp64(g, b->arena, mu, b->owned);
        }
        // autotune: one warm-up run, then one timed run per candidate
        b->shape = cands[0];
        const cudaStream_t bs = b->bs;
        if (cands.size() > 1) {
            batch_time(b, cands[0], bs);
            double best = 1e300;
            for (size_t k = 0; k < cands.size() && k < 16; ++k) {
                const double ms = batch_time(b, cands[k], bs);
                b->tried[k] = cands[k];
                b->tried_ms[k] = ms;
                b->n_tried = (int)k + 1;
                if (ms < best) { best = ms; b->shape = cands[k]; }
            }
        }
        // capture the whole run once
        if (b->use_graph) {
            const uint64_t l0 = nl_kernel_launches();
            NL_CUDA(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
            try {
                batch_enqueue(b, b->shape, bs);
            } catch (NlError &) {
                cudaGraph_t junk = nullptr;
                cudaStreamEndCapture(bs, &junk);
                if (junk) cudaGraphDestroy(junk);
                throw;
            }
            NL_CUDA(cudaStreamEndCapture(bs, &b->graph));
            NL_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
            b->launches_per_run = nl_kernel_launches() - l0;
            nl_uncount_launches(b->launches_per_run);   // captured, not run
        }
    } catch (NlError &e) {
        batch_free(b);
        return e.st;
    }
    *out = b;
    return NL_OK;
}

extern "C" nl_status nl_batch_run(nl_batch *b)
{
    nl_clear_error();
    if (!b) { nl_set_error("NULL argument"); return NL_EINVAL; }
    try {
        cudaStream_t s = b->arena.stream(), bs = b->bs;
        // work queued by the caller before this call comes first
        NL_CUDA(cudaEventRecord(b->join, s));
        NL_CUDA(cudaStreamWaitEvent(bs, b->join, 0));
        ScopedEvent e0, e1;
        NL_CUDA(cudaEventRecord(e0, bs));
        if (b->exec) {
            NL_CUDA(cudaGraphLaunch(b->exec, bs));
            nl_count_launches(b->launches_per_run);
        } else {
            batch_enqueue(b, b->shape, bs);
        }
        NL_CUDA(cudaEventRecord(e1, bs));
        NL_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        NL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        b->last_ms = ms;
        for (nl_system *S : b->sys) S->stats.quadrature_ms = ms;
        // the run's counters (cleared at its start): an approxcaps hull that
        // could not be completed makes the whole run an error
        unsigned long long hs[8];
        NL_CUDA(cudaMemcpy(hs, b->stats, sizeof(hs), cudaMemcpyDeviceToHost));
        if (nl_status st = nl_check_hull_fallbacks(hs[4])) return st;
    } catch (NlError &e) {
        return e.st;
    }
    return NL_OK;
}

extern "C" nl_status nl_batch_system(nl_batch *b, int i, nl_system **out)
{
    nl_clear_error();
    if (!b || !out || i < 0 || i >= (int)b->sys.size()) { nl_set_error("bad argument"); return NL_EINVAL; }
    *out = b->sys[i];
    return NL_OK;
}

extern "C" nl_status nl_batch_get_info(const nl_batch *b, nl_batch_info *info)
{
    nl_clear_error();
    if (!b || !info) { nl_set_error("NULL argument"); return NL_EINVAL; }
    memset(info, 0, sizeof(*info));
    info->n_problems = (int)b->sys.size();
    info->n_groups = (int)b->groups.size();
    info->graph = b->exec ? 1 : 0;
    info->launches_per_run = b->launches_per_run;
    info->last_run_ms = b->last_ms;
    info->units_per_chunk = b->shape.units_per_chunk;
    info->classify_threads = b->shape.classify_threads;
    info->n_tried = b->n_tried;
    for (int k = 0; k < b->n_tried; ++k) {
        info->tried_units_per_chunk[k] = b->tried[k].units_per_chunk;
        info->tried_classify_threads[k] = b->tried[k].classify_threads;
        info->tried_ms[k] = b->tried_ms[k];
    }
    uint64_t np = 0;
    for (nl_system *S : b->sys) np += (uint64_t)S->pairs->npairs;
    info->pairs = np;
    unsigned long long hs[8];
    if (cudaMemcpy(hs, b->stats, sizeof(hs), cudaMemcpyDeviceToHost) == cudaSuccess) {
        info->cut_points = hs[0];
        info->inside_points = hs[1];
        info->mc_samples = hs[2];
        info->mc_accepted = hs[3];
        info->hull_fallbacks = hs[4];
    }
    return NL_OK;
}

extern "C" void nl_batch_destroy(nl_batch *b) { batch_free(b); }
