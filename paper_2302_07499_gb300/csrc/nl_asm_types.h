// Plain argument structures of the assembly launches, shared by the kernel
// translation units and the batch driver (no device code here).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "nl_internal.h"

namespace nla {

// Work is cut into chunks of outer elements so that the per-(pair, point)
// records stay bounded in size.
constexpr int64_t kUnitsPerChunk = int64_t(1) << 25;
// values per event record of the moments (15 used; a multiple of 4 so that
// records start on 16-byte boundaries and read as 16-byte vectors)
constexpr int MQ_STRIDE = 16;
static_assert(MQ_STRIDE % 4 == 0 && MQ_STRIDE >= 15, "moment records are read as 16-byte vectors");

// One problem: its mesh, pairs and pattern (inputs), its outputs, and where
// its outer elements and pairs start in the index space of a launch (0 for a
// single problem; the running sums of the earlier problems in a batch).
struct Prob {
    const double4 *verts;
    const float4 *vhi, *vlo;
    const int4 *tets;
    const uint8_t *in_omega;
    const double *tet_vol;
    const float2 *vol_hl;    // the volumes as float hi + lo
    const int32_t *outer_ids;
    const int32_t *outer_of;
    const double *xq;
    const float *xq_hl;      // [n_outer][4][6] outer points as float hi, lo parts
    const int64_t *pair_ptr;
    const int32_t *pair_tp;
    const int32_t *pair_T;
    const int64_t *rowptr;
    const int32_t *col;
    const int64_t *strip_off;
    double delta2;
    float delta2f;
    double half_gamma;
    int64_t pair_base, outer_base;
    void *D;                 // [npairs][10] staged T'T' moments (R)
    uint8_t *nfull;          // FP32: [npairs] points at which T' is whole (their T'T' part is added in FP64)
    double *Dw;              // FP32 with a kernel shape: [npairs][10] T'T' moments of the whole-T' points (FP64)
    double *strips;          // [strip_total]
    double *TT;              // [n_outer][10]
};

struct AsmArgs {
    Prob self;               // the problem of a single-problem launch
    const Prob *probs;       // batch: the problems (device memory)
    const int32_t *pair_prob;   // batch: problem of every pair of the launch's index space
    const int32_t *outer_prob;  // batch: problem of every outer element
    int64_t o0, o1;          // outer elements of this chunk (launch index space)
    int64_t p0, p1;          // pairs of this chunk (launch index space)
    int max_row;
    int nmc;
    int qmc;                 // fullcaps cap points: 0 Philox draws, 1 shifted Sobol' points
    int hull_maxf;           // face capacity of the approxcaps hull (full capacity except in overflow tests)
    int kpoly;               // 1: kernel shape phi = kc[0] + kc[1] s + kc[2] s^2 + kc[3] s^3 (else phi = 1)
    double kc[4];
    uint32_t rk[20];         // Philox round keys
    // per-chunk work arrays
    uint8_t *uinfo;          // [4*(p1-p0)] vertex-inside mask | 0x10 event | 0x20 zero
    int32_t *evu;            // [4][units] unit of each event, per class (m = 0..3)
    int *nev;                // [5] event count per class; nev[4] = deferred events
    int32_t *fix;            // [units] FP32 approxcaps events deferred to the FP64 pass
    void *Mq;                // [units][MQ_STRIDE] moments (R) of the events, by unit: 15 used, 16-byte aligned records
    unsigned long long *stats;  // [5]
};

// Launch shapes of the quadrature kernels (the batch autotuner varies them).
struct Shape {
    int64_t units_per_chunk = kUnitsPerChunk;
    int classify_threads = 256;
    int events_blocks_per_sm = 0;   // 0: as many as fit
};

// Chunks of whole outer elements over a launch's pair index space; gptr is
// the running pair count at every outer element (n_outer + 1 entries).
inline std::vector<std::pair<int64_t, int64_t>> plan_chunks(const std::vector<int64_t> &gptr, int64_t units,
                                                            int64_t *max_units)
{
    std::vector<std::pair<int64_t, int64_t>> chunks;
    const int64_t no = (int64_t)gptr.size() - 1;
    *max_units = 0;
    for (int64_t o = 0; o < no;) {
        int64_t o1 = o + 1;
        while (o1 < no && 4 * (gptr[o1 + 1] - gptr[o]) <= units) ++o1;
        chunks.push_back({o, o1});
        *max_units = std::max<int64_t>(*max_units, 4 * (gptr[o1] - gptr[o]));
        o = o1;
    }
    return chunks;
}

// ---------------------------------------------------------------------------
// Batch: the problems of one group (same precision, strategy, Monte Carlo
// count and seed) share every launch; each pair and outer element finds its
// problem through pair_prob / outer_prob.  The arithmetic of every unit is
// that of the single-problem launch, so a batched problem's results are
// bitwise those of the problem alone.
struct BatchGroup {
    AsmArgs A;                       // group arguments (probs, maps, work arrays)
    std::vector<int64_t> gptr;       // running pair count over the group's outer elements
    int strategy = 0, precision = 0;
};

inline void philox_round_keys(uint64_t seed, uint32_t rk[20])
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}

inline Prob make_prob(nl_system *sys, void *D, double *strips, double *TT, uint8_t *nfull)
{
    nl_pairs *P = sys->pairs;
    nl_mesh *m = P->mesh;
    Prob r;
    memset(&r, 0, sizeof(r));
    r.verts = m->verts; r.vhi = m->vhi; r.vlo = m->vlo; r.tets = m->tets; r.in_omega = m->in_omega;
    r.tet_vol = m->tet_vol; r.vol_hl = m->vol_hl; r.outer_ids = m->outer_ids; r.outer_of = m->outer_of; r.xq = m->xq;
    r.xq_hl = m->xq_hl;
    r.pair_ptr = P->pair_ptr; r.pair_tp = P->pair_tp; r.pair_T = P->pair_T;
    r.rowptr = P->rowptr; r.col = P->col; r.strip_off = P->strip_off;
    r.delta2 = P->delta * P->delta;
    r.delta2f = (float)r.delta2;
    r.half_gamma = sys->opts.gamma / 2.0;
    r.D = D; r.strips = strips; r.TT = TT; r.nfull = nfull; r.Dw = sys->Dw;
    NL_REQUIRE(r.verts && r.vhi && r.vlo && r.vol_hl && r.tets && r.xq && r.xq_hl && r.pair_ptr && r.pair_tp && r.pair_T &&
                   r.rowptr && r.col && r.strip_off && r.outer_of && r.outer_ids,
               "internal: an input array of the assembly is missing");
    return r;
}

inline void init_group_args(AsmArgs &A, const nl_assemble_opts &o, unsigned long long *stats, int max_row)
{
    A.max_row = max_row;
    A.hull_maxf = nl_hull_max_faces();
    A.nmc = (o.strategy == NL_FULLCAPS || o.strategy == NL_FULLCAPS_QMC) ? o.mc_points : 0;
    A.qmc = o.strategy == NL_FULLCAPS_QMC ? 1 : 0;
    A.kpoly = o.kernel_poly ? 1 : 0;
    for (int k = 0; k < 4; ++k) A.kc[k] = o.kernel_poly ? o.kernel_poly[k] : (k == 0 ? 1.0 : 0.0);
    philox_round_keys(o.seed, A.rk);
    A.stats = stats;
}

}  // namespace nla
