/*
 * wilson_oracle.h -- plain, slow, FP64 CPU oracle for bootstrap AMG on the
 * odd-even reduced 2D Wilson-Dirac system (Brannick & Kahl, "Bootstrap
 * Algebraic Multigrid for the 2D Wilson Dirac system").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that
 * the CUDA library is checked against.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header or table with the CUDA path.
 *
 * Every operator is held as a generic complex CSR matrix built from the
 * paper's definitions with explicit loops; products such as D_eo*D_oe and
 * P^H A P are formed with a textbook sparse product.  Nothing is fused,
 * blocked or reordered beyond what the definitions state.
 *
 * Conventions (all arrays are complex128 = two doubles, re then im):
 *   full lattice site z = y*N + x, unknown index 2*z + s (s = spin 0/1)
 *   gauge U[mu][y][x], mu = 0 (x) or 1 (y); link from (x,y) to (x,y)+e_mu
 *   even/odd half lattice index h = y*(N/2) + x/2 (x+y even resp. odd)
 *   level-l vectors: unknown 2*h + s on the even sublattice of an N_l torus
 */
#ifndef WILSON_ORACLE_H
#define WILSON_ORACLE_H
#include <complex.h>
#include <stdint.h>

typedef double complex cplx;

typedef struct {
  int nrow, ncol, nnz;
  int *rowptr, *col;
  cplx *val;
} or_csr;

enum { OR_ORDER_LEX = 0, OR_ORDER_COLOUR = 1, OR_ORDER_TILE = 2 };

#define OR_MAXLEV 8

typedef struct {
  int L;                 /* number of levels, level 0 = finest (D-hat)      */
  int N[OR_MAXLEV];      /* lattice side of level l (even sublattice)        */
  int B[OR_MAXLEV];      /* cell size from level l to l+1 (0 at coarsest)    */
  int Nfine;
  double m;
  or_csr A[OR_MAXLEV];   /* level operators, 2 n_l x 2 n_l                   */
  or_csr AT[OR_MAXLEV];  /* plain transposes: row i of AT = column i of A    */
  or_csr P[OR_MAXLEV];   /* interpolation level l+1 -> l                     */
  or_csr PH[OR_MAXLEV];  /* P^H                                              */
  or_csr T[OR_MAXLEV];   /* mass matrices T_l = P_l^H P_l (setup only)       */
  int nT;                /* 1 if T is populated                              */
  cplx *lu;              /* coarsest dense LU factors (row major)            */
  int *piv;
  int nc;                /* coarsest dimension                              */
} or_hier;

typedef struct {
  int levels;            /* number of levels (>= 2)                          */
  int block[OR_MAXLEV];  /* cell size per coarsening step (2 or 4)           */
  int k_r, k_e;          /* relaxation / eigen test vectors                  */
  int mu1, mu2;          /* relaxations per visit in setup cycles 1 and 2    */
  int nu_pre, nu_post;   /* solve-cycle smoothing (used by the adaptive step)*/
  int gamma;             /* 1 = V, 2 = W (solve cycle in the adaptive step)  */
  int setup_cycle;       /* 2 = W-cycle setup (Fig. 3.2), 1 = super-V (Sec. 4.2) */
  uint64_t seed;
} or_setup_params;

/* counter-based generator (SplitMix64 output function, Steele/Lea/Flood) */
uint64_t or_rng_u64(uint64_t seed, uint64_t stream, uint64_t i);
cplx or_rng_cgauss(uint64_t seed, uint64_t stream, uint64_t i);

/* ---- operators on the full lattice (Sec. 2) ---- */
int or_wilson_nnz(int N);
int or_wilson_csr(int N, const cplx *U, double m, int *rowptr, int *col, cplx *val);
int or_wilson_apply(int N, const cplx *U, double m, const cplx *psi, cplx *out);
int or_dhat_nnz(int N, const cplx *U, double m);
int or_dhat_csr(int N, const cplx *U, double m, int *rowptr, int *col, cplx *val);
int or_dhat_apply(int N, const cplx *U, double m, const cplx *xe, cplx *ye);
int or_eo_reduce(int N, const cplx *U, double m, const cplx *b, cplx *bhat);
int or_eo_reconstruct(int N, const cplx *U, double m, const cplx *b,
                      const cplx *xe, cplx *psi);

/* ---- level geometry ---- */
int or_colour(int N, int h);
int or_tile_size(int N);
int or_stencil_neighbour(int N, int h, int d);

/* ---- hierarchy ---- */
or_hier *or_hier_import(int N, const cplx *U, double m, int L, const int *Nl,
                        const int *Bl, const cplx *const *Pw,
                        const cplx *const *As);
int or_hier_export(const or_hier *h, cplx *const *Pw, cplx *const *As);
or_hier *or_setup(int N, const cplx *U, double m, const or_setup_params *p,
                  double *ritz_out);
void or_hier_free(or_hier *h);
int or_hier_levels(const or_hier *h, int *Nl, int *Bl);

/* ---- solve-phase steps (Secs. 1, 3.1, 3.5, 4) ---- */
int or_level_apply(const or_hier *h, int l, const cplx *x, cplx *y);
int or_kaczmarz(const or_hier *h, int l, cplx *x, cplx *r, int order,
                int sweeps, double omega, const int *perm);
int or_restrict(const or_hier *h, int l, const cplx *r, cplx *fc);
int or_prolong(const or_hier *h, int l, const cplx *e, cplx *x);
int or_coarsest_solve(const or_hier *h, const cplx *f, cplx *x);
int or_cycle(const or_hier *h, int l, const cplx *f, cplx *x, int nu1, int nu2,
             int gamma, int order);
int or_fgmres(const or_hier *h, const cplx *b, cplx *x, double tol, int mrestart,
              int max_restarts, int nu1, int nu2, int gamma, int precond, int gs_passes,
              int *iters_out, int *restarts_out, double *relres_out);
int or_rho(const or_hier *h, const cplx *x0, double tol, int maxit, int nu1, int nu2,
           int gamma, int order, double *rho_out, int *iters_out, double *hist);
int or_solve(int N, const cplx *U, double m, const or_hier *h, const cplx *b,
             cplx *psi, double tol, int mrestart, int max_restarts, int nu1,
             int nu2, int gamma, int order, int gs_passes, int *iters_out, double *relres_out);

/* ---- setup building blocks (Secs. 3.3-3.5) ---- */
int or_ls_fit(int Nf, int B, int k, const cplx *V, const double *w, cplx *Pw);
int or_galerkin(const or_hier *h, int l, cplx *Ac_stencil);
int or_gen_eig(int n, const cplx *Z, const cplx *T, double *lam, cplx *V);
int or_dense_lu_solve(int n, const cplx *A, const cplx *b, cplx *x);

/* ---- aggregation coarse space (Sec. 4's "more interpolation variables") ----
 * Q [nc][2][B*B][k]: orthonormal columns per (aggregate, spin); Ac
 * [nc][9][2k][2k]: Galerkin block stencil; coarse vectors [nc][2k]. */
int or_agg_interp(int N, int B, int k, const cplx *V, cplx *Q);
int or_agg_galerkin(const or_hier *h, int l, int B, int k, const cplx *Q, cplx *Ac);
int or_agg_apply(int Nc, int k, const cplx *Ac, const cplx *x, cplx *y);
int or_agg_restrict(int N, int B, int k, const cplx *Q, const cplx *r, cplx *fc);
int or_agg_prolong(int N, int B, int k, const cplx *Q, const cplx *e, cplx *x);

/* host threads of this build (1 unless built with OpenMP) */
int or_threads(void);

/* ---- helpers for tests ---- */
int or_csr_dense(const or_csr *A, cplx *dense);
int or_hier_level_dense(const or_hier *h, int l, int which, cplx *dense);

#endif
