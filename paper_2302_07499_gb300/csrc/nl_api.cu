// C-ABI entry points for assembly and the system handle.
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include "nl_internal.h"
#include "nl_quad.cuh"

namespace {

__global__ void k_zero_collar_g(const uint8_t *__restrict__ node_free, double *g, int64_t nv)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv && node_free[i]) g[i] = 0.0;    // only collar values are used
}

}  // namespace

int nl_hull_max_faces()
{
    const char *e = getenv("NL_HULL_MAX_FACES");
    int v = e ? atoi(e) : 0;
    if (v <= 0 || v > nlq::HULL_MAXF) return nlq::HULL_MAXF;
    return v < 8 ? 8 : v;
}

// An assembly whose approxcaps hulls could not all be completed is refused
// (the cells of another strategy would stand in for them).
nl_status nl_check_hull_fallbacks(uint64_t fallbacks)
{
    if (fallbacks == 0) return NL_OK;
    nl_set_error("approxcaps: %llu convex hulls could not be completed within the hull's capacity; the system would "
                 "not be the approxcaps system", (unsigned long long)fallbacks);
    return NL_EGEOM;
}

nl_status nl_check_assemble_opts(const nl_assemble_opts *opts)
{
    if (opts->strategy < NL_NOCAPS || opts->strategy > NL_FULLCAPS_QMC) { nl_set_error("bad strategy"); return NL_EINVAL; }
    if (opts->precision != NL_FP64 && opts->precision != NL_FP32_COMP) { nl_set_error("bad precision"); return NL_EINVAL; }
    if ((opts->strategy == NL_FULLCAPS || opts->strategy == NL_FULLCAPS_QMC) &&
        (opts->mc_points < 1 || opts->mc_points > 4096)) {
        nl_set_error("mc_points must be in 1..4096 for fullcaps");
        return NL_EINVAL;
    }
    if (!isfinite(opts->gamma) || !isfinite(opts->f_const)) { nl_set_error("gamma and f_const must be finite"); return NL_EINVAL; }
    if (opts->g_nodal && opts->g_where != NL_HOST && opts->g_where != NL_DEVICE) { nl_set_error("bad g_where"); return NL_EINVAL; }
    if (opts->f_nodal && opts->f_where != NL_HOST && opts->f_where != NL_DEVICE) { nl_set_error("bad f_where"); return NL_EINVAL; }
    if (opts->kernel_poly) {
        for (int k = 0; k < 4; ++k)
            if (!isfinite(opts->kernel_poly[k])) { nl_set_error("kernel_poly coefficients must be finite"); return NL_EINVAL; }
        if (opts->strategy == NL_APPROXCAPS) {
            nl_set_error("approxcaps takes the constant kernel only (the split of its hull into simplices, "
                         "which the 4-point rule depends on under a kernel shape, is not fixed)");
            return NL_EINVAL;
        }
    }
    return NL_OK;
}

// A system handle with K, A, b, F and the collar values g allocated (g set,
// stream-ordered); throws NlError.
nl_system *nl_system_alloc(nl_pairs *P, const nl_assemble_opts *opts, const nl_device *dev)
{
    nl_mesh *m = P->mesh;
    nl_system *S = new nl_system();
    S->arena.dev = dev ? *dev : P->arena.dev;
    S->pairs = P;
    S->opts = *opts;
    S->opts.g_nodal = nullptr;
    S->opts.f_nodal = nullptr;
    if (opts->kernel_poly) {
        for (int k = 0; k < 4; ++k) S->kernel_c[k] = opts->kernel_poly[k];
        S->opts.kernel_poly = S->kernel_c;
    }
    try {
        cudaStream_t s = S->arena.stream();
        S->K = S->arena.get<double>(P->nnz);
        S->A = S->arena.get<double>(P->nnz_a);
        S->A32 = S->arena.get<float>(P->nnz_a);
        S->L = S->arena.get<double>(std::max<int64_t>(P->nnz_l, 1));
        S->Ap = S->arena.get<double>(std::max<int64_t>(P->ap_slots, 4));
        S->Ap32 = S->arena.get<float>(std::max<int64_t>(P->ap_slots, 4));
        S->b = S->arena.get<double>(m->n_free);
        S->g = S->arena.get<double>(m->nv);
        S->F = S->arena.get<double>(m->nv);
        if (opts->g_nodal) {
            NL_CUDA(cudaMemcpyAsync(S->g, opts->g_nodal, sizeof(double) * m->nv,
                                    opts->g_where == NL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
            { k_zero_collar_g<<<(unsigned)nl_cdiv<int64_t>(m->nv, 256), 256, 0, s>>>(m->node_free, S->g, m->nv); nl_count_launch(); }
            NL_CHECK_LAUNCH();
        } else {
            NL_CUDA(cudaMemsetAsync(S->g, 0, sizeof(double) * m->nv, s));
        }
        if (opts->f_nodal) {
            S->f = S->arena.get<double>(m->nv);
            NL_CUDA(cudaMemcpyAsync(S->f, opts->f_nodal, sizeof(double) * m->nv,
                                    opts->f_where == NL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
        }
    } catch (NlError &) {
        S->arena.release_all();
        delete S;
        throw;
    }
    return S;
}

// nl_assemble with the system's work on the given device / stream (the
// pairs' own when dev is NULL).
nl_status nl_assemble_on(nl_pairs *P, const nl_assemble_opts *opts, const nl_device *dev, nl_system **out)
{
    nl_clear_error();
    if (!P || !opts || !out) { nl_set_error("NULL argument"); return NL_EINVAL; }
    *out = nullptr;
    if (nl_status st = nl_check_assemble_opts(opts)) return st;
    nl_mesh *m = P->mesh;
    nl_system *S = nullptr;
    try {
        S = nl_system_alloc(P, opts, dev);
    } catch (NlError &e) {
        return e.st;
    }
    try {
        cudaStream_t s = S->arena.stream();
        Scratch sc(&S->arena);
        const bool f32 = opts->precision == NL_FP32_COMP;
        void *D = f32 ? (void *)sc.get<float>(10 * P->npairs) : (void *)sc.get<double>(10 * P->npairs);
        double *strips = sc.get<double>(P->strip_total);
        double *TT = sc.get<double>(10 * m->n_outer);
        uint8_t *nfull = f32 ? sc.get<uint8_t>(P->npairs) : nullptr;
        S->Dw = (f32 && S->opts.kernel_poly && S->opts.strategy >= NL_BARYCENTER && S->opts.strategy <= NL_INSIDE)
                    ? sc.get<double>(10 * P->npairs) : nullptr;
        uint64_t *st = sc.get<uint64_t>(8);
        NL_CUDA(cudaMemsetAsync(st, 0, sizeof(uint64_t) * 8, s));
        ScopedEvent ev[3];
        NL_CUDA(cudaEventRecord(ev[0], s));
        if (f32) nl_assemble_fp32(S, (float *)D, strips, TT, nfull, st);
        else nl_assemble_fp64(S, (double *)D, strips, TT, nullptr, st);
        NL_CUDA(cudaEventRecord(ev[1], s));
        nl_reduce_system(S, D, f32 ? 1 : 0, nfull, strips, TT);
        NL_CUDA(cudaEventRecord(ev[2], s));
        NL_CUDA(cudaEventSynchronize(ev[2]));
        S->Dw = nullptr;   // scratch, released with sc
        float ms0 = 0.f, ms1 = 0.f;
        NL_CUDA(cudaEventElapsedTime(&ms0, ev[0], ev[1]));
        NL_CUDA(cudaEventElapsedTime(&ms1, ev[1], ev[2]));
        S->stats.quadrature_ms = ms0;
        S->stats.reduce_ms = ms1;
        uint64_t hs[8];
        NL_CUDA(cudaMemcpyAsync(hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
        NL_CUDA(cudaStreamSynchronize(s));
        S->stats.pairs = (uint64_t)P->npairs;
        S->stats.cut_points = hs[0];
        S->stats.inside_points = hs[1];
        S->stats.mc_samples = hs[2];
        S->stats.mc_accepted = hs[3];
        S->stats.hull_fallbacks = hs[4];
    } catch (NlError &e) {
        S->arena.release_all();
        delete S;
        return e.st;
    }
    if (nl_status st = nl_check_hull_fallbacks(S->stats.hull_fallbacks)) {
        S->arena.release_all();
        delete S;
        return st;
    }
    *out = S;
    return NL_OK;
}

extern "C" nl_status nl_assemble(nl_pairs *P, const nl_assemble_opts *opts, nl_system **out)
{
    return nl_assemble_on(P, opts, nullptr, out);
}

extern "C" void nl_system_destroy(nl_system *S)
{
    if (!S) return;
    S->arena.release_all();
    delete S;
}

extern "C" nl_status nl_system_csr(const nl_system *S, int which, nl_csr_view *out)
{
    nl_clear_error();
    if (!S || !out) { nl_set_error("NULL argument"); return NL_EINVAL; }
    const nl_pairs *P = S->pairs;
    if (which == NL_MAT_K) {
        out->n_rows = P->mesh->nv; out->nnz = P->nnz;
        out->rowptr = P->rowptr; out->col = P->col; out->val = S->K;
    } else if (which == NL_MAT_A) {
        out->n_rows = P->mesh->n_free; out->nnz = P->nnz_a;
        out->rowptr = P->a_rowptr; out->col = P->a_col; out->val = S->A;
    } else if (which == NL_MAT_LIFT) {
        out->n_rows = P->mesh->n_free; out->nnz = P->nnz_l;
        out->rowptr = P->l_rowptr; out->col = P->l_col; out->val = S->L;
    } else {
        nl_set_error("bad matrix selector");
        return NL_EINVAL;
    }
    return NL_OK;
}

extern "C" nl_status nl_system_rhs(const nl_system *S, const double **b, const int32_t **free_nodes)
{
    nl_clear_error();
    if (!S) { nl_set_error("NULL argument"); return NL_EINVAL; }
    if (b) *b = S->b;
    if (free_nodes) *free_nodes = S->pairs->mesh->free_nodes;
    return NL_OK;
}

extern "C" nl_status nl_system_stats(const nl_system *S, nl_assemble_stats *out)
{
    nl_clear_error();
    if (!S || !out) { nl_set_error("NULL argument"); return NL_EINVAL; }
    *out = S->stats;
    return NL_OK;
}
