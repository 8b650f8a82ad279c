/*
 * nlfem — GB300 (sm_103a) assembly and solve of the nonlocal Poisson problem
 * with a constant truncated kernel on P1 tetrahedra, after Chen, Ma & Zhang,
 * "High performance implementation of 3D FEM for nonlocal Poisson problem
 * with different ball approximation strategies".
 *
 * Problem (Sec. 2.1, Eq. nonlocalproblem):  -L u = f in Omega,  u = g on the
 * interaction collar Omega_I, with L u(x) = int_{B_delta(x)} (u(y)-u(x)) gamma dy
 * and a constant gamma inside the ball.  The library assembles the Galerkin
 * system of Eqs. (modified_linear), (Ah), (Fh) with the approximate ball
 * B_{delta,h}(x) of one strategy (Def. nocaps; the simplified 3D approxcaps of
 * Sec. 3.3; fullcaps of Sec. 4.3.2), using the 4-point degree-2 rule for the
 * outer and inner integrals (Sec. 4.3.1), and solves it by conjugate
 * gradients (Alg. 5, last line).
 *
 * Conventions for every call:
 *   - Every call returns an nl_status and never aborts; nl_last_error() gives
 *     a thread-local message for the last failure.
 *   - Host arrays passed in are copied; the caller keeps ownership.  Arrays
 *     flagged NL_DEVICE must be device pointers of the current CUDA device;
 *     they are read on the handle's stream and may be reused once the call
 *     returns (every call that reads caller memory synchronises its stream
 *     before returning).
 *   - Device memory owned by a handle is obtained from nl_device.alloc (or
 *     cudaMalloc when alloc is NULL) and released by the matching destroy.
 *   - All device work runs on nl_device.stream (NULL = legacy default).
 *   - Handles are not thread-safe; use one handle per thread or serialise.
 *   - No call uses the CPU to compute any step of the method: every step
 *     runs in this library's CUDA kernels.  A missing or unusable GPU gives
 *     NL_ECUDA.
 */
#ifndef NLFEM_H
#define NLFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NL_OK = 0,
    NL_EINVAL = 1,      /* bad argument, malformed or inverted mesh */
    NL_ENOMEM = 2,      /* allocator returned NULL */
    NL_ECUDA = 3,       /* CUDA runtime error (message in nl_last_error) */
    NL_ENOTCONV = 4,    /* CG stopped at max_iter above the tolerance */
    NL_ETIMEOUT = 5,    /* a bounded device wait gave up */
    NL_EBUSY = 6,       /* resource limit reached (server queue full) */
    NL_EGEOM = 7        /* a geometric construction of the method failed (an approxcaps
                           hull beyond its capacity); no result is returned */
} nl_status;

/* Ball strategies: the three of Sec. 3.3 / 4.3.2 and the element-level ones of
 * Sec. 4.3 (T' whole or not at all: barycenter - its centroid in the closed
 * ball; overlap - it meets the closed ball; inside - all vertices in the open
 * ball). */
typedef enum {
    NL_NOCAPS = 0,
    NL_APPROXCAPS = 1,
    NL_FULLCAPS = 2,
    NL_BARYCENTER = 3,
    NL_OVERLAP = 4,
    NL_INSIDE = 5,
    /* fullcaps with its cap points from a digitally shifted Sobol' sequence
     * (randomized quasi-Monte Carlo) in place of independent Philox draws:
     * the same cells, the same map from four words to a cell and a point,
     * and the same estimator |S|/N sum 1{|y-x| <= delta}; sample k takes the
     * words of Sobol' point k (Gray-code order, four dimensions, direction
     * numbers from the primitive polynomials x+1, x^2+x+1, x^3+x+1 with
     * Joe & Kuo's initial values) XOR one Philox draw of counter
     * (T, T', q, 0xFFFFFFFF).  Not the paper's method: Sec. 4.3.2 leaves
     * better sampling over the caps open. */
    NL_FULLCAPS_QMC = 6
} nl_strategy;
typedef enum { NL_FP64 = 0, NL_FP32_COMP = 1 } nl_precision;
typedef enum { NL_HOST = 0, NL_DEVICE = 1 } nl_where;
typedef enum { NL_MAT_K = 0, NL_MAT_A = 1, NL_MAT_LIFT = 2 } nl_matrix;

/* Device context: allocator hooks (for example PyTorch's caching allocator)
 * and the stream all work is ordered on.  alloc must return memory usable on
 * the current device, aligned to at least 256 bytes, or NULL. */
typedef struct nl_device {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
    void *stream;                     /* cudaStream_t */
} nl_device;

typedef struct nl_mesh nl_mesh;
typedef struct nl_pairs nl_pairs;
typedef struct nl_system nl_system;

/* ---------------------------------------------------------------------------
 * nl_mesh_create — upload a triangulation of Omega-hat = Omega u Omega_I
 * (Sec. 3.1: conforming, elements of Omega and Omega_I do not straddle dOmega)
 * and precompute per element its volume, centroid, bounding radius and the
 * four quadrature points of the 4-point rule (Sec. 4.3.1).
 *   verts         [nv][3] float64 coordinates.
 *   tets          [nt][4] int32 vertex ids, 0 <= id < nv.
 *   tet_in_omega  [nt] uint8: 1 = element of Omega, 0 = element of the collar.
 *   node_free     [nv] uint8: 1 = node in the open domain Omega (an unknown);
 *                 0 = node in the closed collar, dOmega included (Sec. 3.2),
 *                 where the volume constraint fixes the value.
 *   where         NL_HOST or NL_DEVICE for all four arrays.
 * The folded and the unfolded forms.  The elements marked 1 are the outer
 * elements of the assembly, and a collar element T' (marked 0) carries the
 * weight 2.  So with the true Omega/collar split the assembly is the folded
 * form of Sec. 2.2 (Eqs. weak1 and Ah), whose outer integral runs over Omega
 * only.  Marking every element 1, with node_free unchanged, assembles the
 * unfolded form of Eq. weak0 instead: outer integral over all of Omega-hat,
 * no weight 2.  The load vector then integrates f over every element, and
 * its rows for free nodes are unchanged, because a free node lies in the
 * open Omega and touches no collar element.  So the system (A, b) is that of
 * Eq. weak0.
 * Errors: NL_EINVAL for nv<4, nt<1, an id out of range or an element with
 * non-positive signed volume (vertices must be positively oriented);
 * NL_ENOMEM; NL_ECUDA.  The mesh keeps a pointer to *dev (must outlive it). */
nl_status nl_mesh_create(const nl_device *dev, const double *verts, int64_t nv,
                         const int32_t *tets, int64_t nt, const uint8_t *tet_in_omega,
                         const uint8_t *node_free, int where, nl_mesh **out);
void nl_mesh_destroy(nl_mesh *mesh);

/* nl_mesh_create_box — the Kuhn (Freudenthal) grid of [lo,hi]^3 with `cells`
 * cubes per side and 6 tetrahedra per cube (Sec. 5 uses tetrahedral meshes of
 * Omega-hat = Omega plus its interaction collar), generated on the device:
 * vertex i + (n+1)(j + (n+1)k) at lo + (i,j,k) h with h = (hi-lo)/cells;
 * element 6*cell + p for the p-th permutation of the axes in lexicographic
 * order, vertices (c, c+e_p1, c+e_p1+e_p2, c+(1,1,1)), the last two swapped
 * for the odd permutations so that every element is positively oriented.
 * Omega = [omega_lo, omega_hi]^3, whose bounds must be grid planes: an
 * element belongs to Omega when its cube does, a node is free when it lies
 * strictly inside.  The result is an nl_mesh as from nl_mesh_create.
 * Jitter (a stand-in for the unstructured meshes of Sec. 5): with
 * jitter_frac > 0 every vertex lying on none of the planes of the box and of
 * Omega moves by (2 U_d - 1) * (jitter_frac * h) along axis d, where
 * U_d = (w_d + 1/2) 2^-32 and w = Philox4x32-10 of the counter
 * (vertex id, 0, 0, 0) under the key (seed mod 2^32, seed div 2^32).  Moves
 * are applied class by class over the eight parity classes
 * (i%2 + 2 (j%2) + 4 (k%2) = 0..7), whose vertices share no element; a move
 * is kept only if every element holding the vertex keeps a positive signed
 * volume.  Omega stays exactly [omega_lo, omega_hi]^3.
 * Errors: NL_EINVAL (cells outside 1..1000, hi <= lo, Omega bounds not on
 * grid planes, jitter_frac outside [0, 0.5)), NL_ENOMEM, NL_ECUDA. */
nl_status nl_mesh_create_box(const nl_device *dev, double lo, double hi, int32_t cells, double omega_lo,
                             double omega_hi, double jitter_frac, uint64_t seed, nl_mesh **out);

/* ---------------------------------------------------------------------------
 * nl_pairs_build — element pairs and the fixed sparsity pattern for a horizon
 * delta.  A pair (T, T') has T in Omega and T' any element with
 *     min_q |x_q(T) - T'|^2 <= delta^2
 * over the four quadrature points x_q of T, i.e. T' meets the closed ball
 * around some outer point (the cells kept by Alg. 2).  Pairs are ordered by
 * T (increasing element id), then T'.  The pattern is the union over pairs
 * of (nodes(T) u nodes(T'))^2, symmetric, in CSR with sorted columns.
 * Built once per (mesh, delta) and reused by every strategy.
 * Errors: NL_EINVAL (delta <= 0 or not finite, or more than 65535 columns in
 * one row), NL_ENOMEM, NL_ECUDA.  The pairs keep a pointer to the mesh. */
nl_status nl_pairs_build(nl_mesh *mesh, double delta, nl_pairs **out);
void nl_pairs_destroy(nl_pairs *pairs);

typedef struct {
    int64_t n_vert, n_tet, n_outer;    /* n_outer = elements of Omega */
    int64_t n_pairs;
    int64_t nnz;                       /* pattern of the full matrix K (all nodes) */
    int64_t n_free, nnz_a;             /* unknowns and nnz of A = K[free,free] */
    int32_t max_row;                   /* longest row of K */
    double delta;
    int64_t nnz_lift;                  /* nnz of K[free, collar] */
} nl_pairs_info;
nl_status nl_pairs_get_info(const nl_pairs *pairs, nl_pairs_info *info);

/* Copy the pair list out: outer[n_outer] (element ids of Omega, increasing),
 * ptr[n_outer+1] (int64 offsets), tp[n_pairs] (partner ids).  Any pointer may
 * be NULL to skip it.  where = NL_HOST or NL_DEVICE for the destinations. */
nl_status nl_pairs_export(const nl_pairs *pairs, int32_t *outer, int64_t *ptr, int32_t *tp, int where);

/* ---------------------------------------------------------------------------
 * nl_assemble — stiffness matrix and right-hand side (Alg. 5 with the
 * approximate ball of the chosen strategy).  For every pair and outer point
 * x_q the inner region R = T' n B_{delta,h}(x_q) is:
 *   - T' when all four vertices lie in the open ball;
 *   - nocaps: the convex hull of the inside vertices and the edge/sphere
 *     points (Def. simplex's dividing strategy, Def. nocaps);
 *   - approxcaps: that hull enlarged by the midpoints of the sphere's arcs on
 *     the faces of T' (Sec. 3.3);
 *   - fullcaps: the nocaps cells plus a Monte Carlo estimate over the cap
 *     T' \ hull with mc_points Philox4x32-10 samples keyed by (seed) with
 *     counter (T, T', q, k) (Sec. 4.3.2, Alg. 4).
 * The local contribution is omega*(gamma/2)*|T|/4 * int_R d d^T with
 * d = (-phi_T(x_q), +phi_T'(y)) and omega = 2 when T' is a collar element
 * (Eqs. Ah, replaceBasis), so K (all nodes) is symmetric with zero row sums.
 * With g the nodal volume constraint: A = K[free,free] and
 * b_i = sum_T sum_q w_q phi_i(x_q) f - sum_{j not free} K_ij g_j.
 *   gamma      kernel constant inside the ball (e.g. 15/(2 pi delta^5)).
 *   f_const    constant part of the source f.
 *   g_nodal    [n_vert] nodal values of g (only collar nodes are read);
 *              NULL means g = 0.  g_where: NL_HOST or NL_DEVICE.
 *   f_nodal    [n_vert] nodal values of the rest of the source (only nodes of
 *              elements of Omega are read), or NULL: f = f_const + the P1
 *              interpolant of f_nodal, integrated with the same 4-point rule
 *              (Eq. Fh).  f_where: NL_HOST or NL_DEVICE.
 *   precision  NL_FP64: every step in FP64 (decisions follow a fixed
 *              operation order without fused multiply-add);
 *              NL_FP32_COMP: the per-(pair, point) geometry, Monte Carlo
 *              and moments run in FP32 in coordinates relative to x_q, and
 *              every sum across points, pairs and elements is accumulated in
 *              FP64; matrix entries are FP64.
 * Deterministic: the same inputs give bitwise the same K and b (no floating-
 * point atomics).  Errors: NL_EINVAL (strategy, precision, mc_points outside
 * 1..4096 for fullcaps, gamma not finite), NL_ENOMEM, NL_ECUDA, NL_EGEOM
 * (approxcaps: a hull of the arc midpoints could not be completed within its
 * capacity; no system is returned rather than one with nocaps cells in its
 * place).
 * The environment variable NL_HULL_MAX_FACES (8..24) lowers the hull's face
 * capacity, for tests of that path only.
 *   kernel_poly  non-constant kernels (Sec. 2's gamma(x, y) on the ball,
 *              here gamma phi(|x - y|)): NULL keeps phi = 1 (the constant
 *              kernel above); otherwise 4 finite host doubles c0..c3 (read
 *              during the call) give phi = c0 + c1 s + c2 s^2 + c3 s^3 with
 *              s = min(|x - y|^2 / delta^2, 1) (the element-level strategies
 *              place points past the sphere, where phi keeps its value on
 *              it).  The inner integrals then take the 4-point rule of
 *              Sec. 4.3.1 on every cell and on every whole T', with phi at
 *              the rule points (no longer exact), and every accepted cap
 *              sample is weighted by phi.  Single systems only: the batch
 *              and the server reject a kernel shape (NL_EINVAL), and so does
 *              approxcaps (the rule would depend on how its hull is split
 *              into simplices, which Sec. 3.3 does not fix).  In
 *              NL_FP32_COMP the element-level strategies take whole
 *              elements in FP64, as the constant kernel's closed forms are
 *              taken; nocaps and fullcaps take them, and the cut units,
 *              through FP32 records, and a kernel that vanishes at the
 *              sphere leaves K's far entries small, so their entries are
 *              within 5e-4 rather than 1e-5 (measured: 2.6e-4 at worst,
 *              4.5e-7 at the 99.9th percentile, on a 329,232-element
 *              mesh). */
typedef struct {
    int strategy;            /* nl_strategy */
    int mc_points;           /* fullcaps samples per cap (ignored otherwise) */
    uint64_t seed;           /* Philox key */
    int precision;           /* nl_precision */
    double gamma;
    double f_const;
    const double *g_nodal;
    int g_where;
    const double *f_nodal;   /* NULL: constant f */
    int f_where;
    const double *kernel_poly;  /* NULL: constant kernel; else 4 host doubles, see below */
} nl_assemble_opts;

nl_status nl_assemble(nl_pairs *pairs, const nl_assemble_opts *opts, nl_system **out);
void nl_system_destroy(nl_system *sys);

/* Device views of an assembled matrix (no copy; valid until destroy).
 * NL_MAT_K: full matrix over all nodes (rows/cols = node ids).
 * NL_MAT_A: the free block, rows/cols numbered by increasing node id among
 *           free nodes.
 * NL_MAT_LIFT: K[free, collar], the block that lifts the volume constraint to
 *           the right-hand side (Sec. 2.2: b = F - K[free, collar] g); rows as
 *           for NL_MAT_A, columns = node ids of the collar nodes (sorted). */
typedef struct {
    int64_t n_rows, nnz;
    const int64_t *rowptr;   /* device, n_rows+1 */
    const int32_t *col;      /* device, nnz */
    const double *val;       /* device, nnz */
} nl_csr_view;
nl_status nl_system_csr(const nl_system *sys, int which, nl_csr_view *out);

/* Device pointer to b (n_free doubles) and to the free-node list (n_free int32
 * node ids, increasing). */
nl_status nl_system_rhs(const nl_system *sys, const double **b, const int32_t **free_nodes);

typedef struct {
    uint64_t pairs;            /* element pairs processed */
    uint64_t cut_points;       /* (pair, q) with 1..3 vertices inside */
    uint64_t inside_points;    /* (pair, q) with T' inside the ball */
    uint64_t mc_samples;       /* Monte Carlo samples drawn */
    uint64_t mc_accepted;
    uint64_t hull_fallbacks;   /* approxcaps hulls that fell back to nocaps */
    double quadrature_ms;      /* duration of the quadrature kernel (CUDA events
                                  recorded on the assembly stream around its launch) */
    double reduce_ms;          /* duration of the reduction into K, A and b */
    double classify_ms;        /* the three quadrature kernels, summed over the */
    double events_ms;          /* chunks of pairs: classification, cut-point   */
    double combine_ms;         /* moments (+ Monte Carlo), per-pair combination */
} nl_assemble_stats;
nl_status nl_system_stats(const nl_system *sys, nl_assemble_stats *out);

/* ---------------------------------------------------------------------------
 * nl_solve — conjugate gradients on A u = b from u = 0 (Alg. 5, last line),
 * stopping when ||r||_2 / ||b||_2 <= rtol.
 *   mixed = 0: FP64 CG.
 *   mixed = 1: iterative refinement: r = b - A u in FP64, correction by an
 *              FP32 CG on the FP32 copy of A to inner_rtol, u += d in FP64;
 *              dot products and residuals are FP64 in both modes.
 *   u_out      [n_vert] full nodal solution (free nodes solved, collar nodes
 *              = g), or NULL; where: NL_HOST or NL_DEVICE.
 * Errors: NL_ENOTCONV (info filled, u_out written with the last iterate),
 * NL_EINVAL, NL_ENOMEM, NL_ECUDA. */
typedef struct {
    double rtol;           /* default 1e-12 when <= 0 */
    int max_iter;          /* total inner iterations; default 20000 when <= 0 */
    int mixed;
    double inner_rtol;     /* default 1e-5 when <= 0 */
    int check_every;       /* host polls the residual every k iterations; default 8 */
} nl_solve_opts;

typedef struct {
    int iterations;        /* CG iterations (inner iterations for mixed) */
    int refinements;       /* outer refinement steps (mixed) */
    double rel_residual;   /* final ||b - A u|| / ||b|| in FP64 */
    int barrier_fallbacks; /* systems up to 16384 unknowns run each CG loop in one cooperative
                              launch whose grid barriers wait at most a second (the environment
                              variable NL_CG_BARRIER_WAIT_NS sets another limit, for tests); loops
                              that gave up a wait and were redone with separate launches */
} nl_solve_info;

nl_status nl_solve(nl_system *sys, const nl_solve_opts *opts, double *u_out, int where,
                   nl_solve_info *info);

/* ---------------------------------------------------------------------------
 * nl_solve_static — the FP64 conjugate-gradient solve of nl_solve (mixed is
 * ignored) without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory during
 * the call, e.g. a latency-critical loop that cannot afford cudaMalloc or
 * cudaFree (cudaFree synchronises the whole device), code that runs inside a
 * fixed memory budget reserved up front by another framework, or a thread
 * that holds a lock the caller's allocator may need.
 *   Scratch: the CG vectors live in one fixed device array compiled into the
 *   library (about 5.3 MB, held on every device that loads the library until
 *   the process exits).  Limit: at most 131072 unknowns (n_free); larger
 *   systems get NL_EINVAL with a message.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Sharing: every call uses the same array, which keeps the last call's
 *   contents (each call clears or overwrites what it reads).  Calls whose GPU
 *   work overlaps (other threads, other streams) race on the array; order
 *   them, e.g. on one stream.
 *   u_out: device pointer to n_vert doubles on the current device (or
 *   managed memory; required), written as by nl_solve.  A host pointer gives
 *   NL_EINVAL.  Work runs on the system's stream; the call synchronises it.
 * Errors: NL_EINVAL, NL_ENOTCONV (u_out holds the last iterate), NL_ECUDA. */
nl_status nl_solve_static(nl_system *sys, const nl_solve_opts *opts, double *u_out, nl_solve_info *info);

/* ---------------------------------------------------------------------------
 * Batched assembly (a system layer; the paper has none).  n independent
 * problems, each an nl_pairs with its own options, assembled by shared
 * launches: problems with the same precision, strategy, Monte Carlo count and
 * seed form a group whose (pair, point) units run in one classification, one
 * cut-point and one combination launch per chunk; the reductions into K, A and
 * b follow per problem.  Every unit's arithmetic and every sum's order are
 * those of the problem alone, so each problem's K, A and b are bitwise equal
 * to nl_assemble's.
 *
 * nl_batch_create builds the plan: per problem an nl_system (owned by the
 * batch; nl_batch_system lends it out, valid until nl_batch_destroy), the
 * group maps, and work arrays for the largest chunk.
 *   autotune   1: time candidate launch shapes (units per chunk 2^23, 2^24,
 *              2^25 x classification block 128, 256 threads) on the batch
 *              itself, one run each after a warm-up run, and keep the fastest
 *              (the candidates' timings are in nl_batch_info).  The results of
 *              every run are identical whatever the shape.
 *   use_graph  1: capture one whole run in a CUDA graph that nl_batch_run
 *              replays (the batch's buffers stay fixed).
 * All pairs must share one stream (their nl_device's).  opts: n entries, as
 * for nl_assemble (g_nodal is copied at creation).
 * Errors: NL_EINVAL, NL_ENOMEM, NL_ECUDA. */
typedef struct nl_batch nl_batch;
typedef struct {
    int autotune;
    int use_graph;
    int64_t units_per_chunk;   /* with autotune = 0: the shape to use (0: defaults 2^25 and 256) */
    int classify_threads;
} nl_batch_opts;
nl_status nl_batch_create(nl_pairs *const *pairs, const nl_assemble_opts *opts, int n, const nl_batch_opts *bopts,
                          nl_batch **out);

/* Assemble every problem of the batch (replays the graph when there is one);
 * synchronises the stream before returning.  Errors: NL_EINVAL, NL_ECUDA,
 * NL_EGEOM (an approxcaps hull of some problem could not be completed, as for
 * nl_assemble; the batch's systems are then not valid). */
nl_status nl_batch_run(nl_batch *batch);

/* The system of problem i (the caller's order), owned by the batch.
 * Errors: NL_EINVAL (NULL argument, i out of range). */
nl_status nl_batch_system(nl_batch *batch, int i, nl_system **out);

typedef struct {
    int n_problems, n_groups, graph;
    uint64_t launches_per_run;     /* kernels one run launches */
    double last_run_ms;            /* device time of the last nl_batch_run (CUDA events) */
    int64_t units_per_chunk;       /* the shape in use */
    int classify_threads;
    int n_tried;                   /* autotuner candidates and their run times */
    int64_t tried_units_per_chunk[16];
    int tried_classify_threads[16];
    double tried_ms[16];
    uint64_t pairs, cut_points, inside_points, mc_samples, mc_accepted, hull_fallbacks;   /* last run, summed */
} nl_batch_info;
/* Errors: NL_EINVAL (NULL argument). */
nl_status nl_batch_get_info(const nl_batch *batch, nl_batch_info *info);
void nl_batch_destroy(nl_batch *batch);

/* ---------------------------------------------------------------------------
 * Request server (a system layer; the paper has none): assemble-and-solve
 * requests on Kuhn box meshes, served continuously.  `workers` threads, each
 * with its own stream, take requests first come first served; up to
 * `workers` requests run on the device at once and their kernels overlap.
 * The head of the queue starts when a worker is free and the estimated
 * device footprint of the running requests plus the resident cache plus its
 * own fits budget_bytes (least recently used cache entries that no running
 * request holds are evicted first; a request whose estimate alone exceeds
 * the budget fails with NL_ENOMEM).  With cache = 1 the mesh, pairs and
 * sparsity pattern of a (box, delta) key stay resident between requests.
 * Device memory is stream-ordered (cudaMallocAsync on the worker's stream);
 * the server does not use any nl_device.  Every request runs the
 * single-problem code path, so its result does not depend on what else runs.
 * Times are seconds since nl_server_create (host steady clock). */
typedef struct nl_server nl_server;
typedef struct {
    int64_t budget_bytes;
    int workers;               /* 1..16 */
    int queue_capacity;        /* pending requests; submit beyond it returns NL_EBUSY */
    int cache;
} nl_server_opts;
typedef struct {
    double lo, hi;             /* the box [lo,hi]^3 and its cells per side */
    int32_t cells;
    double omega_lo, omega_hi; /* Omega = [omega_lo, omega_hi]^3 (grid planes) */
    double delta;
    nl_assemble_opts assemble; /* g_nodal and f_nodal must be NULL */
    int g_quadratic;           /* 1: volume constraint g = |x|^2 at the collar nodes; 0: g = 0 */
    nl_solve_opts solve;
    double jitter_frac;        /* vertex jitter of the box mesh (as nl_mesh_create_box; 0: none) */
    uint64_t jitter_seed;
} nl_request;
enum { NL_REQ_QUEUED = 0, NL_REQ_RUNNING = 1, NL_REQ_DONE = 2 };
typedef struct {
    int state;                 /* NL_REQ_* */
    nl_status status;          /* when done: NL_OK, NL_ENOTCONV (u = last iterate) or the error
                                  (NL_EGEOM as for nl_assemble) */
    double t_submit, t_start, t_done;
    double assemble_ms, solve_ms;   /* device time of the assembly and of the solve */
    int64_t n_pairs, n_free, n_vert, est_bytes;
    int iterations, refinements, cache_hit, queue_depth_at_start;
    double rel_residual;
    char message[160];         /* error message when status is an error */
} nl_result;
typedef struct {
    int queued, running, cache_entries;
    int64_t cache_bytes, running_bytes;
} nl_server_load;
/* Errors: NL_EINVAL (NULL argument; workers outside 1..16, budget <= 0 or
 * queue capacity < 1), NL_ECUDA (no device, stream creation).  *out is NULL
 * on error. */
nl_status nl_server_create(const nl_server_opts *opts, nl_server **out);
/* Queue a request (copied); the ticket names it until nl_server_release.
 * Errors: NL_EINVAL (NULL argument, cells < 1, delta not positive and
 * finite, hi <= lo, g_nodal set), NL_EBUSY (queue_capacity requests
 * pending).  Device errors of the request itself arrive in its result. */
nl_status nl_server_submit(nl_server *server, const nl_request *req, uint64_t *ticket);
/* The request's state and result so far (never blocks).  Errors: NL_EINVAL
 * (NULL argument, unknown ticket). */
nl_status nl_server_poll(nl_server *server, uint64_t ticket, nl_result *res);
/* Wait until the request is done (timeout_s <= 0: no limit; NL_ETIMEOUT
 * otherwise), then copy its result and, when u_out is not NULL, its nodal
 * solution (n_vert doubles, host memory of n_u >= n_vert entries).
 * Errors: NL_EINVAL (NULL server, unknown ticket, n_u too small),
 * NL_ETIMEOUT.  The request's own status is res->status. */
nl_status nl_server_wait(nl_server *server, uint64_t ticket, double timeout_s, nl_result *res, double *u_out,
                         int64_t n_u);
/* Forget a finished request (NL_EBUSY while it is queued or running;
 * NL_EINVAL for an unknown ticket). */
nl_status nl_server_release(nl_server *server, uint64_t ticket);
/* Errors: NL_EINVAL (NULL argument). */
nl_status nl_server_get_load(nl_server *server, nl_server_load *out);
/* Stops the workers after their current requests; queued ones are dropped. */
void nl_server_destroy(nl_server *server);

/* ---------------------------------------------------------------------------
 * Diagnostic entry points (not on the assembly path).  Host arrays in and
 * out; they run on the default stream with their own temporary device
 * buffers and synchronise before returning.
 *
 * nl_probe_moments — the inner moments of the approximate ball for n single
 * cases (element T' with vertices tets_xyz[c][4][3], outer point x[c][3],
 * Philox counter words ids[c] = (T, T', q)), computed by the same device code
 * as nl_assemble.  moments[c][15] = (|R|, int_R lambda'_a (a=0..3),
 * int_R lambda'_a lambda'_b for (a,b) = (0,0) (0,1) (0,2) (0,3) (1,1) (1,2)
 * (1,3) (2,2) (2,3) (3,3)), lambda' the barycentric coordinates of T'.
 * Definitions as for nl_assemble (Def. nocaps, Sec. 3.3, Sec. 4.3.2).
 * Errors: NL_EINVAL, NL_ECUDA. */
nl_status nl_probe_moments(const double *tets_xyz, const double *x, const uint32_t *ids, int64_t n,
                           double delta, int strategy, int mc_points, uint64_t seed, int precision,
                           double *moments);

/* nl_probe_mc_samples — the fullcaps Monte Carlo samples of n single cases
 * (T' vertices tets_xyz[c][4][3], outer point x[c][3], Philox counter words
 * ids[c] = (T, T', q)), drawn by the same device code as nl_assemble's
 * fullcaps events (Sec. 4.3.2, Alg. 4): per case n_samples[c] = mc_points,
 * or 0 when T' has no cap for x (all vertices inside, or T' not meeting the
 * closed ball); per sample k (arrays [n][mc_points], row-major):
 * cell[c][k] the cap cell the sample fell in (-1 past n_samples[c]),
 * accepted[c][k] = 1 when |y - x|^2 <= delta^2, y[c][k][3] the point.
 * NL_FP64: the points of the arithmetic specification (global coordinates,
 * no fused multiply-add).  NL_FP32_COMP: the FP32 path's decisions and its
 * FP32 point relative to x, returned as x + that offset.  At most 2^20 cases.
 * Errors: NL_EINVAL (NULL pointer, mc_points outside 1..4096, precision),
 * NL_ECUDA. */
nl_status nl_probe_mc_samples(const double *tets_xyz, const double *x, const uint32_t *ids, int64_t n, double delta,
                              int mc_points, uint64_t seed, int precision, int32_t *n_samples, int32_t *cell,
                              uint8_t *accepted, double *y);

/* nl_probe_qmc_samples — as nl_probe_mc_samples for NL_FULLCAPS_QMC: the
 * cap points of the shifted Sobol' sequence (see nl_strategy). */
nl_status nl_probe_qmc_samples(const double *tets_xyz, const double *x, const uint32_t *ids, int64_t n,
                               double delta, int mc_points, uint64_t seed, int precision, int32_t *n_samples,
                               int32_t *cell, uint8_t *accepted, double *y);

/* nl_probe_philox — Philox4x32-10 (Salmon et al., SC'11) of n counters
 * ctr[n][4] under the key (key & 0xffffffff, key >> 32): the generator that
 * draws the fullcaps Monte Carlo points.  out[n][4].  Errors: NL_EINVAL,
 * NL_ECUDA. */
nl_status nl_probe_philox(const uint32_t *ctr, uint64_t key, int64_t n, uint32_t *out);

/* nl_spmv_time — device time of one SpMV y = A x of the CG (the kernel
 * nl_solve runs for systems above 16384 unknowns: A's rows padded to
 * multiples of 4 entries, 8 lanes per row, 16-byte loads) on the system's
 * free block A, FP64 values or the FP32 copy, with the partials of x.y,
 * after one untimed launch (CUDA events on the system's stream):
 *   flush_bytes = 0: averaged over `reps` back-to-back launches (as in the
 *     CG, where A may partly stay in L2);
 *   flush_bytes > 0: each of `reps` launches timed alone after a write of
 *     flush_bytes bytes to a scratch buffer (more than the L2 size evicts A:
 *     the HBM-bound time).
 * bytes_per_spmv (optional): the algorithmic traffic nnz (value + column
 * index) + rowptr + x + y.  Errors: NL_EINVAL, NL_ENOMEM, NL_ECUDA. */
nl_status nl_spmv_time(nl_system *sys, int precision, int reps, int64_t flush_bytes, double *ms_per_spmv,
                       double *bytes_per_spmv);

/* nl_probe_alu_rates — measured ALU throughput of the current device, the
 * denominators of the quadrature kernels' ALU roofline (no part of the
 * paper's method).  Each entry is operations per second of one
 * register-only microbenchmark (independent chains, 8 blocks of 256 threads
 * per SM, best of 3 runs timed with CUDA events on the default stream):
 *   [0] FP32 fused multiply-add   [1] FP64 fused multiply-add
 *   [2] 32-bit mad.lo             [3] 32-bit mul.hi
 *   [4] 3-input xor, counted as 2 operations
 *   [5] Philox4x32-10 draws, 80 operations each
 *   [6] the fullcaps sample of Sec. 4.3.2 (a Philox draw, the cell choice,
 *       three uniforms, their sort, the spacings, the point and the ball
 *       test), 121 operations each, with its cell in registers.
 * n must be at least 7.  Takes a few tens of milliseconds; synchronises the
 * device.  Errors: NL_EINVAL, NL_ECUDA. */
nl_status nl_probe_alu_rates(double *ops_per_s, int n);

/* Thread-local message of the last failing call (empty string if none). */
const char *nl_last_error(void);

/* Number of kernels this library has launched in this process (all entry
 * points, all threads); for launch accounting around a timed region. */
uint64_t nl_kernel_launches(void);

/* Library version string. */
const char *nl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NLFEM_H */
