/* CPU FP64 oracle (test infrastructure only; see nl_oracle.c). */
#ifndef NL_ORACLE_H
#define NL_ORACLE_H
#include <stdint.h>

#define OR_NOCAPS 0
#define OR_APPROXCAPS 1
#define OR_FULLCAPS 2
#define OR_BARYCENTER 3
#define OR_OVERLAP 4
#define OR_INSIDE 5
/* fullcaps with the cap points from a digitally shifted Sobol' sequence
 * instead of independent Philox draws (randomized quasi-Monte Carlo) */
#define OR_FULLCAPS_QMC 6

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_tet_volume(const double v[12]);
void or_quad_points(const double v[12], double xq[12]);
double or_dist2_point_tet(const double p[3], const double v[12]);
int or_pair_predicate(const double vT[12], const double vTp[12], double delta);
int64_t or_pairs(const double *verts, int64_t nv, const int32_t *tets, int64_t nt,
                 const uint8_t *in_omega, double delta, int use_grid,
                 const int32_t *outer_list, int64_t n_list,
                 int64_t *ptr_out, int32_t *tp_out, int64_t cap);
int or_hull_tets(int n, const double *p, double *out, int maxout);
int or_hull_tets_labeled(int n, const double *p, const unsigned *lab, double *out, int maxout);
void or_mc_point(const double *S, int ns, const uint32_t u[4], double y[3], int *which);
void or_qmc_point(const double *S, int ns, const uint32_t u[4], double y[3], int *which);
int or_region_moments(const double vTp[12], const double x[3], double delta, int strategy,
                      int nmc, uint64_t seed, uint32_t idT, uint32_t idTp, uint32_t q,
                      const double *kpoly, double M[15], double *mc_vol);
int or_cap_samples(const double vTp[12], const double x[3], double delta, int nmc, uint64_t seed,
                   uint32_t idT, uint32_t idTp, uint32_t q, double *y, int32_t *cell, uint8_t *accepted);
int or_cap_samples_qmc(const double vTp[12], const double x[3], double delta, int nmc, uint64_t seed,
                       uint32_t idT, uint32_t idTp, uint32_t q, double *y, int32_t *cell, uint8_t *accepted);
void or_sobol_point(uint32_t k, uint32_t out[4]);
int or_pair_block(const double vT[12], const double vTp[12], double delta, double gamma,
                  int tp_in_collar, int strategy, int nmc, uint64_t seed,
                  uint32_t idT, uint32_t idTp, const double *kpoly, double blk[64]);
int64_t or_assemble_blocks(const double *verts, const int32_t *tets, const uint8_t *in_omega,
                           double delta, double gamma, int strategy, int nmc, uint64_t seed,
                           const double *kpoly, const int32_t *pT, const int32_t *pTp, int64_t npairs,
                           double *blocks, int nthreads);
void or_load_vector(const double *verts, const int32_t *tets, int64_t nt, const uint8_t *in_omega,
                    int64_t nv, double fconst, const double *fnodal, double *F);
int or_num_threads(void);
#endif
