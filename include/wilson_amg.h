/*
 * wilson_amg.h -- C ABI of the GB300 (sm_103a) bootstrap-AMG solver for the
 * odd-even reduced 2D Wilson-Dirac system.
 *
 * Method: J. Brannick and K. Kahl, "Bootstrap Algebraic Multigrid for the 2D
 * Wilson Dirac system".  The problem is D psi = b (Sec. 1, Eq. 1.1) with the
 * 2D Wilson matrix D = D_0 + m I (Sec. 2, Eq. 2.1; N_s = 2 spins, U(1)
 * links).  The library reduces it to the even-site Schur complement
 * Dhat = I - D_eo D_oe (Sec. 3.2, Eq. 3.2), solves Dhat psi_e = bhat with
 * FGMRES preconditioned by an AMG cycle (Kaczmarz smoothing, Sec. 3.1;
 * least-squares interpolation P and Galerkin restriction P^H, Secs. 3.3 and
 * 3.5; a direct coarsest solve, Sec. 4), and reconstructs psi_o.
 *
 * Conventions (every pointer is a DEVICE pointer unless it says "host"):
 *   complex numbers are complex128 (two doubles, re then im) at this ABI;
 *   lattice side L (= N): L >= 16, L a power of two (so L/16 is one);
 *   gauge  U[2][L][L]  (mu, y, x): U_mu(x, y) on the edge (x,y) -> (x,y)+e_mu,
 *          mu = 0 is x, mu = 1 is y; gauge links are periodic;
 *   D acts as (D psi)(z) = (m+2) psi(z) - 1/2 sum_mu [(1 - s_mu) U_mu(z)
 *          psi(z+mu) + (1 + s_mu) conj(U_mu(z-mu)) psi(z-mu)], s_mu the
 *          Pauli matrices, with an extra factor -1 on hops across the y
 *          boundary (antiperiodic fermions in y);
 *   full fields  [nrhs][L][L][2]  (rhs, y, x, spin);
 *   level vectors [nrhs][n_l][2] with n_l = N_l^2/2 sites of the even
 *          sublattice of an N_l x N_l torus, site h <-> y = h / (N_l/2),
 *          x = 2 (h mod N_l/2) + (y mod 2);  level 0 is the fine even grid.
 *   Interpolation weights [n_l][2][4] (site, spin, cell corner k = ka+2kb)
 *   and coarse stencils [n_l][9][2][2] (site, offset d = 3(da+1)+(db+1) in
 *   rotated coordinates a = (x+y)/2, b = (x-y)/2, row spin, column spin)
 *   are the layouts of the hierarchy file (see amg_export).
 *
 * Ownership: the caller owns every array it passes; the library copies the
 * gauge in wilson_create and owns its hierarchy and workspace.  Streams:
 * each wl_op runs its kernels on a work stream of its own, which at every
 * call first waits (an event) for the work already queued on the stream
 * given to wilson_create, so device arrays produced there are ready.  Calls
 * that return results to the host (amg_solve, amg_fgmres, amg_rho, the
 * per-step entry points) synchronise the work stream before returning.
 *
 * Errors: 0 = OK, 1 = WL_NOT_CONVERGED (x holds the best iterate), negative
 * values are errors; wl_last_error() returns a message for the calling
 * thread.  No call faults the device on bad arguments: sizes, levels and
 * pointers are checked on the host first (WL_EINVAL).
 */
#ifndef WILSON_AMG_H
#define WILSON_AMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wl_op wl_op;   /* Wilson operator for one gauge field          */
typedef struct wl_amg wl_amg; /* AMG hierarchy (cached setup) for one wl_op   */

enum {
  WL_OK = 0,
  WL_NOT_CONVERGED = 1,
  WL_EINVAL = -1,
  WL_OOM = -2,
  WL_ECUDA = -3,
  WL_TIMEOUT = -4,       /* a kernel's bounded wait for its own asynchronous copies or
                            tensor-core work ran out (one second); the call's results
                            are not valid.  No kernel waits on another kernel or rank
                            (the one grid-wide barrier is a cooperative launch's). */
  WL_NAN = -5,
  WL_BAD_HIERARCHY = -6
};

enum { WL_FP64 = 0, WL_FP32 = 1, WL_FP32_BF16 = 2 }; /* cycle precision */
enum { WL_OP_D = 0, WL_OP_DHAT = 1, WL_OP_Z = 2 };    /* wl_apply        */
enum { WL_CYCLE_V = 0, WL_CYCLE_W = 1 };

typedef struct {
  int levels;             /* number of grids, >= 2; the coarsest is solved directly */
  int block[8];           /* cell size (2 or 4) of coarsening step l -> l+1          */
  int k_r, k_e;           /* relaxation / eigenvector test vectors (Sec. 3.4)        */
  int setup_mu[2];        /* Kaczmarz sweeps per visit, setup cycles 1 and 2 (Sec. 4.1) */
  int nu_pre, nu_post;    /* solve-cycle smoothing sweeps                           */
  double omega;           /* Kaczmarz relaxation weight (1 = the paper's)           */
  int cycle;              /* WL_CYCLE_V or WL_CYCLE_W                                */
  int fgmres_m;           /* FGMRES restart length (<= 32)                          */
  int max_restarts;
  int precision;          /* WL_FP64, WL_FP32 or WL_FP32_BF16 (cycle arithmetic)    */
  unsigned long long seed;/* seed of the setup's random test vectors                */
  int gs_passes;          /* Gram-Schmidt passes (1 = CGS, 2 = CGS with one reorth.) */
  int zero_guess;         /* 1: amg_solve ignores the contents of x                 */
  int sweep_kernel;       /* Kaczmarz launch form: 0 = autotuned (before the first
                             cycle of a batch width is captured, every form of one
                             sweep is timed on each level and the fastest kept; until
                             then, or for per-step calls, a heuristic), 1 = one launch
                             per colour, 2 = one cooperative launch per level visit.
                             Every form computes the same numbers in the same order. */
  int kacz_order;         /* Kaczmarz ordering: 0 = 16 colours (a mod 4, b mod 4) over the
                             whole grid; 1 = tile-coloured: 8x8 tiles in (a, b) with four
                             tile colours, the 16 colours inside each tile (grids with
                             N >= 64; smaller grids keep order 0).  Both are forward
                             sweeps over a permutation of the variables (Sec. 3.1). */
  int arnoldi_matvec;     /* precision of the Arnoldi matvec w = Dhat z_j inside a
                             restart cycle: 0 = FP64 (matrix-free from the links), 1 =
                             FP32 when the cycle is FP32 or BF16 (the FP32 copy of the
                             9-point Dhat stencil, result widened to FP64 for the
                             Gram-Schmidt).  The true residual at every restart
                             stays FP64, so the accuracy is unchanged; a cycle whose
                             Arnoldi relation holds to FP32 rounding may need one more
                             restart. */
  int setup_cycle;        /* bootstrap setup cycles: 0 = W-cycle (Fig. 3.2), 1 = super-V
                             (Sec. 4.2: each grid visited once, mu 2^l relaxations
                             before and after the coarse visit on grid l, one coarsest
                             eigensolve per setup cycle) */
  int overlap;            /* 1: amg_solve splits a batch of at least 32 right-hand sides
                             into two halves solved at the same time on two streams (a
                             second workspace and graph set that share the hierarchy's
                             operators, made on first use), so that one half's
                             Gram-Schmidt runs beside the other half's cycle.  Each
                             right-hand side computes what it computes alone (results
                             agree with overlap = 0 up to the rounding of batch-width-
                             dependent reductions). */
  int gs_arith;           /* arithmetic of the Gram-Schmidt process (the Krylov basis,
                             its dots, updates and norms): 0 = FP64; 1 = double-float,
                             each value an unevaluated sum of two floats (about 48
                             significant bits) computed on the FP32 pipes with
                             error-free transformations; the restart update x += Z y
                             sums Z y the same way and adds it to x in FP64; the
                             Hessenberg matrix and Givens rotations stay FP64.  Requires
                             an FP32 or BF16 cycle with arnoldi_matvec = 1 (EINVAL
                             otherwise).  The true residual at every restart stays
                             FP64, so the accuracy a solve reaches is unchanged. */
} amg_params;

typedef struct {
  int status;             /* WL_OK, WL_NOT_CONVERGED or WL_NAN for this right-hand side */
  int restarts;           /* FGMRES cycles run                                       */
  int iters;              /* FGMRES iterations (preconditioner applications)         */
  double true_relres;     /* ||bhat - Dhat x|| / ||bhat|| recomputed in FP64         */
} wl_info;

/* Fill *p with the defaults: V(2,2) cycle, FGMRES(20), k_r = k_e = 8, setup
 * relaxation 10 then 5 (Sec. 4.1), FP64, CGS with one reorthogonalisation. */
void amg_params_default(amg_params *p);

/* Create the Wilson operator D = D_0 + m I of Eq. 2.1 for the gauge field
 * `gauge` (device, complex128 [2][L][L], copied).  cuda_stream is a
 * cudaStream_t (NULL = default stream).  m must satisfy m + 2 != 0.
 * Errors: WL_EINVAL (L not a power of two >= 16, NULL pointers), WL_OOM,
 * WL_ECUDA. */
int wilson_create(const void *gauge, int L, double m, void *cuda_stream, wl_op **out);
void wl_destroy(wl_op *op);

/* y = D x (which = WL_OP_D; x, y full fields [nrhs][L][L][2]), y = Z x
 * with Z = Gamma5 D (which = WL_OP_Z, Thm. 3.1; Gamma5 = +1 on spin 0, -1 on
 * spin 1, so Z is Hermitian; same layout) or
 * y = Dhat x (which = WL_OP_DHAT, Eq. 3.2 with the 1/c scaling of Sec. 3.2;
 * x, y level-0 vectors [nrhs][L^2/2][2]), computed matrix-free from the
 * links in precision prec (WL_FP64 or WL_FP32; FP32 rounds x and the links
 * to float and accumulates in float).  Errors: WL_EINVAL. */
int wl_apply(wl_op *op, int which, const void *x, void *y, int nrhs, int prec);

/* Sec. 3.2, two-step solve: bhat = b_e/c - (D_eo/c)(b_o/c) with c = m + 2
 * (b full fields, bhat level-0 vectors), and psi_e = x_e,
 * psi_o = b_o/c - (D_oe/c) x_e.  Errors: WL_EINVAL. */
int wl_eo_reduce(wl_op *op, const void *b, void *bhat, int nrhs);
int wl_eo_reconstruct(wl_op *op, const void *b, const void *xe, void *psi, int nrhs);

/* Bootstrap setup (Secs. 3.4-3.5, 4.1) on the GPU: W-cycle setup with
 * setup_mu[0] sweeps, an adaptive step, a second W-cycle with setup_mu[1]
 * sweeps; least-squares interpolation (Eq. 3.4) and Galerkin coarse
 * operators P^H D P on every level; coarsest operator inverted in FP64.
 * Errors: WL_EINVAL (levels / blocks incompatible with L), WL_OOM, WL_ECUDA. */
int amg_setup(wl_op *op, const amg_params *params, wl_amg **out);

/* Solve D psi = b for nrhs right-hand sides (b, x full fields
 * [nrhs][L][L][2], device).  x is the initial guess unless
 * params.zero_guess.  Stops each right-hand side when its FP64 relative
 * residual of the reduced system is <= tol, or after max_restarts FGMRES
 * cycles (x then holds the last iterate, whose true residual info reports).
 * info: host array [nrhs].  A right-hand side whose residual becomes
 * non-finite (a NaN or Inf in its b or initial guess, say) is retired with
 * info[r].status = WL_NAN and its x is not meaningful; the other right-hand
 * sides of the batch are solved as usual (no kernel mixes right-hand sides).
 * Returns WL_NAN if some right-hand side was retired that way, else
 * WL_NOT_CONVERGED if some missed tol, else WL_OK; other negative values
 * are errors of the whole call. */
int amg_solve(wl_amg *amg, const void *b, void *x, int nrhs, double tol, wl_info *info);

/* amg_solve with b and x in host memory (same layout, same results bit for
 * bit).  Each batch of up to 256 right-hand sides is copied into device
 * staging buffers held with the hierarchy (2 x batch x L x L x 2 complex
 * doubles, allocated on first use, freed by amg_free), solved, and copied
 * back; with params.overlap the two lanes copy their own halves on their
 * own streams, so one lane's copies run beside the other lane's solve.
 * Page-locked host memory (cudaHostAlloc, cudaHostRegister) lets the copies
 * run asynchronously; pageable memory works, with synchronous copies.  The
 * call returns when x is written.  Errors and statuses as amg_solve, plus
 * WL_OOM for the staging buffers. */
int amg_solve_host(wl_amg *amg, const void *b, void *x, int nrhs, double tol, wl_info *info);

/* Hierarchy file: header "WLAMGH01", version, levels, N_l, B_l, m, gauge
 * checksum, interpolation weights of every non-coarsest level and coarse
 * stencils of levels >= 1 (complex128, layouts above), FNV-1a 64 checksum.
 * amg_import rebuilds a hierarchy for `op` from such a file (its solve
 * parameters from *params, NULL = defaults); WL_BAD_HIERARCHY if the file
 * is corrupt or belongs to another gauge field / mass. */
int amg_export(wl_amg *amg, const char *path);
int amg_import(wl_op *op, const char *path, const amg_params *params, wl_amg **out);
/* FNV-1a 64 (offset basis 14695981039346656037, prime 1099511628211) of n
 * host bytes at p: the hierarchy file's checksum and the gauge identity
 * wilson_create records.  Host only (no GPU needed); 0 for p = NULL with
 * n > 0. */
unsigned long long wl_hash_bytes(const void *p, size_t n);
void amg_destroy(wl_amg *amg);

/* Number of levels and the lattice side of level l (host outputs). */
int amg_levels(wl_amg *amg, int *N_out /* host [levels] */);

/* ---- per-step entry points of the solve phase (used by the parity tests) ----
 * Vectors are level-l vectors [nrhs][n_l][2] in FP64 at this ABI; prec
 * selects the arithmetic of the step (WL_FP64, WL_FP32, WL_FP32_BF16).     */

/* y = A_l x, A_0 = Dhat (explicit 9-point stencil), A_l = P^H A_{l-1} P. */
int amg_level_apply(wl_amg *amg, int level, const void *x, void *y, int nrhs, int prec);
/* `sweeps` multicolour Kaczmarz sweeps (Sec. 3.1) on A_l x = f with the
 * residual r = f - A_l x carried along; x, r updated in place. */
int amg_kaczmarz(wl_amg *amg, int level, void *x, void *r, int nrhs, int sweeps, int prec);
/* fc = P_l^H r (level l -> l+1) and x += P_l e (level l+1 -> l). */
int amg_restrict(wl_amg *amg, int level, const void *r, void *fc, int nrhs, int prec);
int amg_prolong(wl_amg *amg, int level, const void *e, void *x, int nrhs, int prec);
/* x = A_L^{-1} f on the coarsest level (FP64 inverse). */
int amg_coarsest(wl_amg *amg, const void *f, void *x, int nrhs);
/* One preconditioning cycle x = M(f) on level 0 from x = 0 (the
 * configured V or W cycle, nu_pre / nu_post sweeps). */
int amg_cycle(wl_amg *amg, const void *f, void *x, int nrhs, int prec);
/* FGMRES on Dhat x = bhat (level-0 vectors, x = initial guess); info host
 * array [nrhs].  Return values and per-right-hand-side status as for
 * amg_solve. */
int amg_fgmres(wl_amg *amg, const void *bhat, void *x, int nrhs, double tol, wl_info *info);
/* Sec. 4's convergence estimate of the stand-alone solver: the configured
 * cycle (V or W, nu_pre / nu_post, precision) used as the stationary
 * iteration x <- x + M(0 - Dhat x) on Dhat x = 0, Dhat in FP64, so the
 * iterate is the error e.  From e^0 = x0 (level-0 vectors [nrhs][L^2/2][2],
 * device) it runs until |e^nu| <= tol |e^0| for every right-hand side or
 * nu = maxit; rho[r] = |e^nu| / |e^(nu-1)| at the right-hand side's own
 * stopping nu (iters[r]).  rho, iters: host [nrhs]; hist: host
 * [nrhs][maxit + 1] or NULL, |e^k| for k <= iters[r] (rest untouched).
 * x (device, same layout) receives the error after the batch's last
 * iteration.  A right-hand side whose error norm overflows (a divergent
 * cycle) stops there, keeping the ratio of its last two finite norms.
 * Returns WL_OK if every right-hand side met tol, WL_NOT_CONVERGED
 * otherwise; WL_EINVAL for nrhs outside 1..256, tol < 0 or maxit < 1. */
int amg_rho(wl_amg *amg, const void *x0, void *x, int nrhs, double tol, int maxit, double *rho, int *iters,
            double *hist);

/* y = Dhat x in FP64 with no device allocation (the paper has no counterpart;
 * this is a service of the library).  For callers that cannot allocate device
 * memory when they need the operator: a process whose device memory is
 * already held by its own pool (a framework's caching allocator, say, so a
 * raw cudaMalloc would fail), or a latency-critical loop that cannot afford
 * the device-wide synchronisation cudaMalloc / cudaFree imply.  The odd-site
 * intermediate lives in a fixed 16 MiB device array of the library
 * (2^20 complex doubles, held on every GPU that loads the library until the
 * process exits); the call allocates nothing, not even through torch.
 * x, y: device, level-0 vectors [nrhs][L^2/2][2] complex128, caller-owned.
 * Limit: L^2 * nrhs <= 2^20 (for example L = 512 with nrhs <= 4, L = 1024
 * with nrhs = 1); larger sizes return WL_EINVAL with a message naming the
 * limit.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it for the life of the process, so the
 * library must not be used across a cudaDeviceReset (or any teardown of the
 * device's primary context): the cached address would then be stale.  All
 * calls share the array, which keeps the last call's contents (every
 * element read is first overwritten, so nothing needs clearing); calls whose
 * work overlaps on the GPU race on it.  Synchronous: the call waits for its
 * kernels (a stream synchronisation) and returns after y is written, so it
 * must not be called while the caller's stream, or the operator's, is being
 * captured into a CUDA graph. */
int wl_dhat_apply_noalloc(wl_op *op, const void *x, void *y, int nrhs);

/* ---- aggregation coarse space (Sec. 4: "more interpolation variables") ----
 * Sec. 4 names, as the alternative it did not explore, coarse spaces with
 * more interpolation variables per coarse point.  An aggregation coarse
 * space of level `level` of a hierarchy: every B x B cell of the full
 * coarsening (B = 2 or 4, cells in the rotated coordinates a = (x+y)/2,
 * b = (x-y)/2) is an aggregate; per aggregate and spin the k test vectors V
 * restricted there are orthonormalised by modified Gram-Schmidt in their
 * given order, giving k columns of P per spin (2k coarse variables per coarse
 * site, Gamma5 P = P Gamma5c).  The Galerkin operator Ac = P^H A_l P (Sec.
 * 3.5) is a 9-point stencil of dense 2k x 2k complex blocks on the N_l / B
 * lattice.
 * Layouts (device, complex128): V [k][n_l][2] (level-l vectors); Q
 * [nc][2][B*B][k] (coarse site, spin, member ia B + ib of the cell, column);
 * Ac [nc][9][2k][2k] (site, offset d as for the stencils above, row variable
 * s k + kappa, column variable t k + lambda); coarse vectors [nrhs][nc][2k].
 * Requirements: N_l / B >= 8, 1 <= k <= min(16, B^2); WL_EINVAL otherwise, or
 * when V restricted to some (aggregate, spin) has rank < k.  The object keeps
 * its hierarchy alive. */
typedef struct wl_agg wl_agg;
enum { WL_AGG_FP64 = 0, WL_AGG_FP32 = 1, WL_AGG_TC = 2, WL_AGG_TC1 = 3 }; /* agg_apply kernels */
int agg_create(wl_amg *amg, int level, int B, int k, const void *V, wl_agg **out);
/* the same from given Q and Ac (device, layouts above), e.g. an exported one */
int agg_import(wl_amg *amg, int level, int B, int k, const void *Q, const void *Ac, wl_agg **out);
int agg_export(wl_agg *g, void *Q, void *Ac);
/* number of coarse sites, coarse lattice side and k (host outputs, each may be NULL) */
int agg_info(wl_agg *g, int *nc, int *Nc, int *k);
void agg_destroy(wl_agg *g);
/* y = Ac x for nrhs right-hand sides (x, y coarse vectors, caller-owned):
 * kernel WL_AGG_FP64 (CUDA cores, FP64), WL_AGG_FP32 (CUDA cores, FP32
 * arithmetic on FP32 copies of Ac and x) or WL_AGG_TC (k = 8 only: the
 * tensor cores, tcgen05.mma on TF32 operands split into high and low parts,
 * FP32 accumulation, accurate to FP32 rounding) or WL_AGG_TC1 (k = 8: the
 * tensor cores on the TF32-rounded operands alone, one product per term,
 * about 1e-3 relative; exact to FP32 accumulation when Ac and x are TF32
 * numbers).  1 <= nrhs <= 4096.
 * WL_TIMEOUT if a tensor-core wait ran out (the kernel then stops early and
 * y is not valid).  Synchronous. */
int agg_apply(wl_agg *g, const void *x, void *y, int nrhs, int kernel);
/* fc = P^H r and x += P e (r, x level-l vectors; fc, e coarse vectors), FP64. */
int agg_restrict(wl_agg *g, const void *r, void *fc, int nrhs);
int agg_prolong(wl_agg *g, const void *e, void *x, int nrhs);
/* average duration (host output, ms) of one apply kernel launch for nrhs
 * right-hand sides on the object's internal buffers, over reps launches
 * (CUDA events on the library's work stream) */
int agg_time_apply(wl_agg *g, int nrhs, int kernel, int reps, double *avg_ms);

/* ---- serving: continuous batching over resident hierarchies ----
 * A server keeps hierarchies of several gauge fields (lattice sizes may
 * differ) resident and answers solve requests.  srv_add reserves, for each
 * hierarchy, a number of right-hand-side slots (max_slots_per_config, halved
 * until the workspace fits the remaining device-memory budget; WL_OOM when
 * not even one slot fits).  A worker thread per hierarchy admits queued
 * right-hand sides into free slots at every FGMRES restart boundary, runs one
 * restart cycle for the packed active slots on that hierarchy's work stream,
 * and retires right-hand sides whose true FP64 relative residual reaches the
 * request's tol, reconstructing their solution into the request's x.  So
 * work of different hierarchies overlaps on the device and requests join
 * while others run.  A right-hand side's arithmetic does not depend on its
 * batch mates (all reductions are per right-hand side), so its result alone
 * and in a mix agree up to the rounding of the reduction trees.
 * Pointers b, x of srv_submit: device, full fields [nrhs][L][L][2] of the
 * hierarchy's lattice, caller-owned, ready (synchronised) before the call and
 * untouched by the caller until srv_poll reports the request done.  A
 * hierarchy added to a server must not be used by other calls while the
 * server runs.  srv_poll's latency is host wall time from srv_submit to the
 * retirement of the request's last right-hand side.  srv_start captures the
 * cycle graph of every packed width (1 .. slots) of every hierarchy before
 * the workers start, so no stream capture runs while clients work and
 * clients may synchronise the whole device. */
typedef struct wl_server wl_server;
int srv_create(unsigned long long hbm_budget_bytes, int max_slots_per_config, wl_server **out);
int srv_add(wl_server *srv, wl_amg *amg, int *cfg_id);
/* Slots reserved for configuration cfg and the device bytes they hold. */
int srv_info(wl_server *srv, int cfg, int *slots, unsigned long long *bytes);
int srv_start(wl_server *srv);
int srv_submit(wl_server *srv, int cfg, const void *b, void *x, int nrhs, double tol, long long *req_id);
/* *done = 1 once every right-hand side of the request is retired; returns
 * the request's status (WL_OK, WL_NOT_CONVERGED, or WL_NAN when one of its
 * right-hand sides had a non-finite residual: that one alone is retired,
 * other requests and the server go on). */
int srv_poll(wl_server *srv, long long req_id, int *done, wl_info *info /* host [nrhs] */, double *latency_ms);
int srv_drain(wl_server *srv);
void srv_destroy(wl_server *srv);

/* ---- instrumentation (benchmarks, tests) ---- */
enum {
  WL_K_DHAT = 0,      /* matrix-free FP64 Dhat apply (two hop kernels)       */
  WL_K_KACZ = 1,      /* one colour pass of the Kaczmarz sweep on `level`     */
  WL_K_STENCIL = 2,   /* residual r = f - A_l x on `level`                    */
  WL_K_RESTRICT = 3,  /* P^H from `level` to level + 1                        */
  WL_K_PROLONG = 4,   /* P from level + 1 to `level`                          */
  WL_K_COARSEST = 5,  /* dense FP64 coarsest solve                            */
  WL_K_GS_DOT = 6,    /* FP64 multi-dot of 11 Krylov vectors (Gram-Schmidt)   */
  WL_K_GS_AXPY = 7,   /* FP64 multi-axpy of 11 Krylov vectors                 */
  WL_K_KACZ_TILE = 8, /* one tile-colour launch (a quarter of a tile-coloured sweep) on `level` */
  WL_K_FP64_FMA = 9   /* not an operator kernel: the FP64 FMA throughput of the device, 8 blocks
                         of 256 threads per SM, each thread 8 independent chains of 4096
                         dependent FMAs (2 flop each); level, nrhs and prec are checked as for
                         the other kinds and otherwise unused */
};
/* Average duration (host output, milliseconds) of one launch of kernel
 * family `kind` in the launch configuration the solver uses for `nrhs`
 * right-hand sides and cycle precision `prec`, timed with CUDA events on
 * the library's work stream over `reps` back-to-back launches on the
 * hierarchy's own work buffers (their contents are not preserved).
 * Errors: WL_EINVAL. */
int wl_time_kernel(wl_amg *amg, int kind, int level, int nrhs, int prec, int reps, double *avg_ms);
/* Kaczmarz launch form used on `level` (not the coarsest) for `nrhs`
 * right-hand sides in precision `prec`: form 0 = one launch per colour,
 * 1 = cooperative launch with *param blocks, 2 = tile-coloured kernel with
 * right-hand-side chunk (*param & 255) and right-hand sides per thread
 * ((*param >> 8) & 15: 1 or 2; 8 = one per thread with paired FP32 FMAs);
 * bit 0x1000: the persistent form (r double-buffered by bulk copies); bit
 * 0x2000: each (site, right-hand side) split over a pair of lanes, one per
 * spin component (FP32, paired FMAs); 3 = one launch for all colours with a block per
 * (*param & 255) right-hand sides (small levels, x and r in shared memory; bit 0x100: the stencil
 * rows and denominators in shared memory too); *us = the autotuner's measured time of one
 * sweep in microseconds, 0 when the form was not measured (explicit
 * sweep_kernel, or no cycle of that width yet).  Errors: WL_EINVAL. */
int amg_sweep_form(wl_amg *amg, int level, int nrhs, int prec, int *form, int *param, float *us);
/* Pin the Kaczmarz launch form of `level` (not the coarsest) for `nrhs`
 * right-hand sides in precision `prec` (form and param as in
 * amg_sweep_form; the form must belong to the hierarchy's ordering on that
 * level).  The autotuner then keeps it, so a cycle of that width captured
 * afterwards uses it; graphs captured earlier are not changed.  For
 * reproducible measurements (a profiler slows every launch, so the tuner's
 * timings under it do not hold).  Ignored while sweep_kernel != 0.  Not
 * thread-safe against solves on the same hierarchy.  Errors: WL_EINVAL. */
int amg_pin_sweep_form(wl_amg *amg, int level, int nrhs, int prec, int form, int param);
/* amg_kaczmarz with an explicit launch form (form and param as reported by
 * amg_sweep_form; the form must belong to the hierarchy's ordering on that
 * level), for tests and measurements: every form of one ordering computes
 * the same numbers.  Errors: WL_EINVAL (no such form). */
int amg_kaczmarz_form(wl_amg *amg, int level, void *x, void *r, int nrhs, int sweeps, int prec, int form, int param);
/* Number of kernels this library has launched in this process (a captured
 * graph counts each of its kernel nodes at every replay). */
long long wl_launch_count(void);

/* Last error message of the calling thread ("" if none). */
const char *wl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
