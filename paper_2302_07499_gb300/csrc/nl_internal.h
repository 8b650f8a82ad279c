// Internal declarations of the nlfem CUDA library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nlfem.h"

// ---------------------------------------------------------------------------
// error plumbing: every entry point returns nl_status; the message is kept
// per thread.
void nl_set_error(const char *fmt, ...);
void nl_clear_error();
// process-wide count of kernels this library launched (nl_kernel_launches)
void nl_count_launch();

struct NlError {
    nl_status st;
};

#define NL_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t _e = (call);                                                       \
        if (_e != cudaSuccess) {                                                       \
            nl_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(_e)); \
            throw NlError{NL_ECUDA};                                                   \
        }                                                                              \
    } while (0)

#define NL_CHECK_LAUNCH() NL_CUDA(cudaGetLastError())

#define NL_REQUIRE(cond, ...)                                                          \
    do {                                                                               \
        if (!(cond)) {                                                                 \
            nl_set_error(__VA_ARGS__);                                                 \
            throw NlError{NL_EINVAL};                                                  \
        }                                                                              \
    } while (0)

// A timing event destroyed with its scope, so a call that throws between
// creating and reading it does not leak it.
struct ScopedEvent {
    cudaEvent_t e = nullptr;
    ScopedEvent() { NL_CUDA(cudaEventCreate(&e)); }
    ~ScopedEvent()
    {
        if (e) cudaEventDestroy(e);
    }
    ScopedEvent(const ScopedEvent &) = delete;
    ScopedEvent &operator=(const ScopedEvent &) = delete;
    operator cudaEvent_t() const { return e; }
};

// Device allocations owned by a handle; released in reverse order.
struct DevArena {
    nl_device dev{};
    std::vector<void *> ptrs;
    void *raw(size_t bytes);
    template <class T> T *get(size_t n) { return static_cast<T *>(raw(sizeof(T) * (n ? n : 1))); }
    void release(void *p);
    void release_all();
    cudaStream_t stream() const { return static_cast<cudaStream_t>(dev.stream); }
};

// Scratch that lives for one call (freed on scope exit).
struct Scratch {
    DevArena *arena;
    std::vector<void *> mine;
    explicit Scratch(DevArena *a) : arena(a) {}
    template <class T> T *get(size_t n) {
        T *p = arena->get<T>(n);
        mine.push_back(p);
        return p;
    }
    ~Scratch() {
        for (size_t i = mine.size(); i-- > 0;) arena->release(mine[i]);
    }
};

struct nl_mesh {
    DevArena arena;
    int64_t nv = 0, nt = 0, n_outer = 0, n_free = 0;
    double4 *verts = nullptr;      // x, y, z, 0
    float4 *vhi = nullptr;         // float hi part of the coordinates
    float4 *vlo = nullptr;         // float lo part (coordinate - hi, rounded)
    float2 *vol_hl = nullptr;      // element volumes as float hi + lo
    int4 *tets = nullptr;
    uint8_t *in_omega = nullptr;
    uint8_t *node_free = nullptr;
    double4 *tet_cr = nullptr;     // centroid xyz, bounding radius
    double *tet_vol = nullptr;
    int32_t *outer_ids = nullptr;  // Omega elements, increasing id
    int32_t *outer_of = nullptr;   // element -> outer index or -1
    double *xq = nullptr;          // [n_outer][4][3] quadrature points
    float *xq_hl = nullptr;        // [n_outer][4][6] the same as float hi xyz, lo xyz
    int32_t *free_idx = nullptr;   // node -> free index or -1
    int32_t *free_nodes = nullptr; // [n_free]
    int64_t *ne_ptr = nullptr;     // node -> incident elements (sorted), packed elem<<2|local
    int32_t *ne_ent = nullptr;
    double rmax = 0.0;
    double bbmin[3] = {0, 0, 0}, bbmax[3] = {0, 0, 0};
};

struct nl_pairs {
    DevArena arena;
    nl_mesh *mesh = nullptr;
    double delta = 0.0;
    int64_t npairs = 0;
    int64_t *pair_ptr = nullptr;   // [n_outer+1]
    int32_t *pair_tp = nullptr;    // [npairs]
    int32_t *pair_T = nullptr;     // [npairs] element id of the outer element
    int64_t *tp_ptr = nullptr;     // [nt+1] pairs having the element as T'
    int32_t *tp_pair = nullptr;    // [npairs] pair ids, increasing
    int64_t nnz = 0;
    int64_t *rowptr = nullptr;     // [nv+1]
    int32_t *col = nullptr;        // [nnz]
    int32_t *perm = nullptr;       // [nnz] position of the transposed entry
    int32_t *elem_pos = nullptr;   // [nt][16] positions of the element block, -1 if inactive
    int64_t *strip_off = nullptr;  // [n_outer*4+1]
    int64_t strip_total = 0;
    int32_t max_row = 0;
    int64_t max_pairs_per_outer = 0;
    int64_t nnz_a = 0;
    int64_t *a_rowptr = nullptr;   // [n_free+1]
    int32_t *a_col = nullptr;      // [nnz_a]
    int32_t *a_src = nullptr;      // [nnz_a] position in K
    // A's rows padded to multiples of 4 entries (the CG's SpMV reads 16-byte
    // vectors): row r holds entries [4 ap_rowptr4[r], 4 ap_rowptr4[r+1]);
    // a pad has column r and no source (value 0)
    int64_t ap_slots = 0;
    int64_t *ap_rowptr4 = nullptr; // [n_free+1] in units of 4 entries
    int32_t *ap_col = nullptr;     // [ap_slots]
    int32_t *ap_src = nullptr;     // [ap_slots] position in A, or -1 for a pad
    int64_t nnz_l = 0;             // L = K[free, collar]
    int64_t *l_rowptr = nullptr;   // [n_free+1]
    int32_t *l_col = nullptr;      // [nnz_l] collar node ids
    int32_t *l_src = nullptr;      // [nnz_l] position in K
};

struct nl_system {
    DevArena arena;
    nl_pairs *pairs = nullptr;
    nl_assemble_opts opts{};
    double kernel_c[4] = {1.0, 0.0, 0.0, 0.0};   // the kernel shape's coefficients (opts.kernel_poly points here)
    double *Dw = nullptr;          // FP32-comp with a kernel shape, during assembly: [npairs][10] T'T' moments
                                   // of the points at which T' is whole, in FP64
    double *K = nullptr;           // [nnz]
    double *A = nullptr;           // [nnz_a]
    float *A32 = nullptr;          // [nnz_a]
    double *L = nullptr;           // [nnz_l] values of K[free, collar]
    double *Ap = nullptr;          // [ap_slots] A's values in the padded rows
    float *Ap32 = nullptr;         // [ap_slots] the same in FP32
    double *b = nullptr;           // [n_free]
    double *g = nullptr;           // [nv]
    double *F = nullptr;           // [nv]
    double *f = nullptr;           // [nv] nodal source values (NULL: f is the constant f_const only)
    nl_assemble_stats stats{};
};

// ---------------------------------------------------------------------------
// shared device utilities (nl_util.cu)
void nl_exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, DevArena *arena, cudaStream_t s);
// out[i] = sum_{j<i} in[j] for i in [0,n], out has n+1 entries; returns out[n] (synchronises)
int64_t nl_scan_counts(const int64_t *counts, int64_t *out, int64_t n, DevArena *arena, cudaStream_t s);
// sort the int32 keys of each segment [ptr[i], ptr[i+1]) ascending; max_seg = longest segment
void nl_segmented_sort_i32(int32_t *keys, const int64_t *ptr, int64_t nseg, int64_t max_seg,
                           DevArena *arena, cudaStream_t s);
int nl_num_sms();

// kernels of other translation units
nl_status nl_pairs_build_impl(nl_mesh *mesh, double delta, nl_pairs **out);
void nl_assemble_fp64(nl_system *sys, double *D, double *strips, double *TT, uint8_t *nfull, uint64_t *stats);
void nl_assemble_fp32(nl_system *sys, float *D, double *strips, double *TT, uint8_t *nfull, uint64_t *stats);
// nfull (FP32 only, else NULL): per pair, the points at which T' is whole
void nl_reduce_system(nl_system *sys, const void *D, int d_is_float, const uint8_t *nfull, const double *strips,
                      const double *TT);
void nl_reduce_system_into(nl_system *sys, const void *D, int d_is_float, const uint8_t *nfull, const double *strips,
                           const double *TT, double *G, double *E, cudaStream_t s);
nl_status nl_check_hull_fallbacks(uint64_t fallbacks);
// Face capacity of the approxcaps hull: the full capacity unless the
// environment variable NL_HULL_MAX_FACES (a testing knob for the overflow
// path) asks for less; never below the 8 faces of the starting polytope.
int nl_hull_max_faces();
nl_status nl_check_assemble_opts(const nl_assemble_opts *opts);
nl_system *nl_system_alloc(nl_pairs *P, const nl_assemble_opts *opts, const nl_device *dev = nullptr);
nl_status nl_assemble_on(nl_pairs *P, const nl_assemble_opts *opts, const nl_device *dev, nl_system **out);
void nl_count_launches(uint64_t n);
void nl_uncount_launches(uint64_t n);
namespace nla { struct BatchGroup; struct Shape; }
void nl_batch_alloc_work_fp32(nla::BatchGroup &g, DevArena &arena, int64_t max_units, std::vector<void *> &owned);
void nl_batch_alloc_work_fp64(nla::BatchGroup &g, DevArena &arena, int64_t max_units, std::vector<void *> &owned);
void nl_batch_launch_fp32(const nla::BatchGroup &g, const nla::Shape &sh, cudaStream_t s);
void nl_batch_launch_fp64(const nla::BatchGroup &g, const nla::Shape &sh, cudaStream_t s);
nl_status nl_solve_impl(nl_system *sys, const nl_solve_opts *opts, double *u_out, int where,
                        nl_solve_info *info);

template <class T> static inline T nl_cdiv(T a, T b) { return (a + b - 1) / b; }
