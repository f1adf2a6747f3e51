/*
 * wilson_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Brannick & Kahl, "Bootstrap Algebraic Multigrid for the 2D Wilson Dirac
 * system".  Each function names the section / equation it restates.  The
 * CUDA library is checked against this file; the two share no code.
 *
 * Readings of passages that the paper leaves open are marked "Reading:".
 *
 * The file builds two ways.  The plain build (gcc, no OpenMP) is the oracle
 * that the tests check against.  The all-cores build (-fopenmp) is timed as
 * the CPU baseline only: its "#pragma omp" lines split loops whose
 * iterations are independent (matrix rows, the sites of one Kaczmarz colour,
 * the tiles of one tile colour, vector updates) over the host cores; the
 * plain build ignores them, so its arithmetic is the serial one.
 */
#include "wilson_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ESTRUCT (-3)

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: the SplitMix64 output function (Steele,    */
/* Lea & Flood 2014) applied to a counter.  u64(seed, stream, i) =          */
/* sm(sm(sm(seed) + stream) + i), sm(z) = mix13(z + 0x9E3779B97F4A7C15).     */
/* Complex Gaussian: Box-Muller on two uniforms in (0,1].                    */
/* ------------------------------------------------------------------------ */
static uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t or_rng_u64(uint64_t seed, uint64_t stream, uint64_t i) {
  return sm64(sm64(sm64(seed) + stream) + i);
}

static double u01(uint64_t u) { return ((double)(u >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

/* Sec. 4: test vectors "normal distribution, expectation zero, variance one";
 * Reading: real and imaginary parts are independent N(0,1). */
cplx or_rng_cgauss(uint64_t seed, uint64_t stream, uint64_t i) {
  double u1 = u01(or_rng_u64(seed, stream, 2 * i));
  double u2 = u01(or_rng_u64(seed, stream, 2 * i + 1));
  double r = sqrt(-2.0 * log(u1));
  double t = 2.0 * M_PI * u2;
  return r * cos(t) + I * (r * sin(t));
}

/* ------------------------------------------------------------------------ */
/* Generic complex CSR matrices.                                            */
/* ------------------------------------------------------------------------ */
static void csr_free(or_csr *A) {
  free(A->rowptr);
  free(A->col);
  free(A->val);
  memset(A, 0, sizeof(*A));
}

typedef struct {
  int n, cap;
  int *r, *c;
  cplx *v;
} triplets;

static int trip_push(triplets *t, int r, int c, cplx v) {
  if (t->n == t->cap) {
    int nc = t->cap ? 2 * t->cap : 1024;
    int *nr = realloc(t->r, sizeof(int) * nc);
    if (!nr) return OR_ENOMEM;
    t->r = nr;
    int *ncol = realloc(t->c, sizeof(int) * nc);
    if (!ncol) return OR_ENOMEM;
    t->c = ncol;
    cplx *nv = realloc(t->v, sizeof(cplx) * nc);
    if (!nv) return OR_ENOMEM;
    t->v = nv;
    t->cap = nc;
  }
  t->r[t->n] = r;
  t->c[t->n] = c;
  t->v[t->n] = v;
  t->n++;
  return OR_OK;
}

static void trip_free(triplets *t) {
  free(t->r);
  free(t->c);
  free(t->v);
  memset(t, 0, sizeof(*t));
}

/* rows sorted by column, duplicate entries summed */
static int csr_from_triplets(int nrow, int ncol, const triplets *t, or_csr *A) {
  memset(A, 0, sizeof(*A));
  A->nrow = nrow;
  A->ncol = ncol;
  int *cnt = calloc((size_t)nrow + 1, sizeof(int));
  if (!cnt) return OR_ENOMEM;
  for (int k = 0; k < t->n; ++k) cnt[t->r[k] + 1]++;
  for (int i = 0; i < nrow; ++i) cnt[i + 1] += cnt[i];
  int *col = malloc(sizeof(int) * (t->n ? t->n : 1));
  cplx *val = malloc(sizeof(cplx) * (t->n ? t->n : 1));
  int *fill = malloc(sizeof(int) * ((size_t)nrow + 1));
  if (!col || !val || !fill) {
    free(cnt); free(col); free(val); free(fill);
    return OR_ENOMEM;
  }
  memcpy(fill, cnt, sizeof(int) * ((size_t)nrow + 1));
  for (int k = 0; k < t->n; ++k) {
    int p = fill[t->r[k]]++;
    col[p] = t->c[k];
    val[p] = t->v[k];
  }
  free(fill);
  /* insertion sort each row, then merge duplicates */
  int *rp = malloc(sizeof(int) * ((size_t)nrow + 1));
  if (!rp) { free(cnt); free(col); free(val); return OR_ENOMEM; }
  int out = 0;
  rp[0] = 0;
  for (int i = 0; i < nrow; ++i) {
    int b = cnt[i], e = cnt[i + 1];
    for (int p = b + 1; p < e; ++p) {
      int c = col[p];
      cplx v = val[p];
      int q = p - 1;
      while (q >= b && col[q] > c) {
        col[q + 1] = col[q];
        val[q + 1] = val[q];
        q--;
      }
      col[q + 1] = c;
      val[q + 1] = v;
    }
    for (int p = b; p < e; ++p) {
      if (out > rp[i] && col[out - 1] == col[p]) {
        val[out - 1] += val[p];
      } else {
        col[out] = col[p];
        val[out] = val[p];
        out++;
      }
    }
    rp[i + 1] = out;
  }
  free(cnt);
  A->rowptr = rp;
  A->col = col;
  A->val = val;
  A->nnz = out;
  return OR_OK;
}

static void csr_matvec(const or_csr *A, const cplx *x, cplx *y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < A->nrow; ++i) {
    cplx s = 0;
    for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) s += A->val[p] * x[A->col[p]];
    y[i] = s;
  }
}

/* adj = 0: plain transpose, adj = 1: conjugate transpose */
static int csr_transpose(const or_csr *A, int adj, or_csr *T) {
  triplets t = {0};
  for (int i = 0; i < A->nrow; ++i)
    for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
      int rc = trip_push(&t, A->col[p], i, adj ? conj(A->val[p]) : A->val[p]);
      if (rc) { trip_free(&t); return rc; }
    }
  int rc = csr_from_triplets(A->ncol, A->nrow, &t, T);
  trip_free(&t);
  return rc;
}

/* C = A * B, row by row with a dense accumulator */
static int csr_mul(const or_csr *A, const or_csr *B, or_csr *C) {
  if (A->ncol != B->nrow) return OR_EINVAL;
  cplx *acc = calloc((size_t)B->ncol, sizeof(cplx));
  int *mark = malloc(sizeof(int) * (size_t)B->ncol);
  int *list = malloc(sizeof(int) * (size_t)B->ncol);
  if (!acc || !mark || !list) { free(acc); free(mark); free(list); return OR_ENOMEM; }
  for (int j = 0; j < B->ncol; ++j) mark[j] = -1;
  triplets t = {0};
  int rc = OR_OK;
  for (int i = 0; i < A->nrow && !rc; ++i) {
    int nl = 0;
    for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
      int k = A->col[p];
      for (int q = B->rowptr[k]; q < B->rowptr[k + 1]; ++q) {
        int j = B->col[q];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0;
          list[nl++] = j;
        }
        acc[j] += A->val[p] * B->val[q];
      }
    }
    for (int q = 0; q < nl && !rc; ++q) rc = trip_push(&t, i, list[q], acc[list[q]]);
  }
  if (!rc) rc = csr_from_triplets(A->nrow, B->ncol, &t, C);
  trip_free(&t);
  free(acc); free(mark); free(list);
  return rc;
}

int or_csr_dense(const or_csr *A, cplx *dense) {
  memset(dense, 0, sizeof(cplx) * (size_t)A->nrow * A->ncol);
  for (int i = 0; i < A->nrow; ++i)
    for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
      dense[(size_t)i * A->ncol + A->col[p]] += A->val[p];
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2, Eq. (2.1) in two dimensions (N_s = 2, N_c = 1, U(1) links):       */
/*   (D psi)_z = (m + 2) psi_z                                              */
/*      - 1/2 sum_mu [ (1 - s_mu) U_mu(z) psi_{z+mu}                        */
/*                   + (1 + s_mu) conj(U_mu(z-mu)) psi_{z-mu} ]             */
/* with s_1, s_2 the Pauli matrices.  Reading: the paper's gamma_2 is        */
/* -sigma_2; the Pauli sigma_2 is used (the spectrum is the same).  The      */
/* boundary is periodic in x and antiperiodic in y: a hop across y = N-1 ->  */
/* 0 (either direction) carries a factor -1.                                */
/* ------------------------------------------------------------------------ */
static void pauli(int mu, cplx s[2][2]) {
  if (mu == 0) {
    s[0][0] = 0; s[0][1] = 1;
    s[1][0] = 1; s[1][1] = 0;
  } else {
    s[0][0] = 0; s[0][1] = -I;
    s[1][0] = I; s[1][1] = 0;
  }
}

static int wilson_triplets(int N, const cplx *U, double m, triplets *t) {
  int rc = OR_OK;
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
      int z = y * N + x;
      for (int s = 0; s < 2 && !rc; ++s) rc = trip_push(t, 2 * z + s, 2 * z + s, m + 2.0);
      for (int mu = 0; mu < 2 && !rc; ++mu) {
        cplx sg[2][2];
        pauli(mu, sg);
        /* forward neighbour z + mu */
        int xf = (mu == 0) ? (x + 1) % N : x;
        int yf = (mu == 1) ? (y + 1) % N : y;
        double bf = (mu == 1 && y == N - 1) ? -1.0 : 1.0;
        cplx uf = U[(size_t)mu * N * N + (size_t)y * N + x];
        /* backward neighbour z - mu; link U_mu(z - mu) */
        int xb = (mu == 0) ? (x + N - 1) % N : x;
        int yb = (mu == 1) ? (y + N - 1) % N : y;
        double bb = (mu == 1 && y == 0) ? -1.0 : 1.0;
        cplx ub = U[(size_t)mu * N * N + (size_t)yb * N + xb];
        int zf = yf * N + xf, zb = yb * N + xb;
        for (int s = 0; s < 2 && !rc; ++s)
          for (int tt = 0; tt < 2 && !rc; ++tt) {
            cplx id = (s == tt) ? 1.0 : 0.0;
            cplx vf = -0.5 * (id - sg[s][tt]) * uf * bf;
            cplx vb = -0.5 * (id + sg[s][tt]) * conj(ub) * bb;
            if (vf != 0) rc = trip_push(t, 2 * z + s, 2 * zf + tt, vf);
            if (!rc && vb != 0) rc = trip_push(t, 2 * z + s, 2 * zb + tt, vb);
          }
      }
    }
  return rc;
}

static int wilson_matrix(int N, const cplx *U, double m, or_csr *D) {
  triplets t = {0};
  int rc = wilson_triplets(N, U, m, &t);
  if (!rc) rc = csr_from_triplets(2 * N * N, 2 * N * N, &t, D);
  trip_free(&t);
  return rc;
}

int or_wilson_nnz(int N) { return N >= 3 ? 2 * N * N * 9 : -1; } /* 1 + 4 hops x 2 entries per row */

int or_wilson_csr(int N, const cplx *U, double m, int *rowptr, int *col, cplx *val) {
  or_csr D;
  int rc = wilson_matrix(N, U, m, &D);
  if (rc) return rc;
  memcpy(rowptr, D.rowptr, sizeof(int) * ((size_t)D.nrow + 1));
  memcpy(col, D.col, sizeof(int) * (size_t)D.nnz);
  memcpy(val, D.val, sizeof(cplx) * (size_t)D.nnz);
  int nnz = D.nnz;
  csr_free(&D);
  return nnz;
}

int or_wilson_apply(int N, const cplx *U, double m, const cplx *psi, cplx *out) {
  or_csr D;
  int rc = wilson_matrix(N, U, m, &D);
  if (rc) return rc;
  csr_matvec(&D, psi, out);
  csr_free(&D);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: odd-even reduction.  With even points numbered first,           */
/* D = [[D_ee, D_eo], [D_oe, D_oo]], D_ee = D_oo = c I (c = m + 2), and      */
/* after scaling by 1/c the Schur complement is Eq. (3.2):                  */
/*   Dhat = I - (D_eo / c)(D_oe / c).                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  or_csr Deo, Doe; /* already scaled by 1/c */
  double c;
} eo_blocks;

static int half_index(int N, int x, int y) { return y * (N / 2) + x / 2; }

static int eo_split(int N, const cplx *U, double m, eo_blocks *eb) {
  if (N < 2 || N % 2) return OR_EINVAL;
  or_csr D;
  int rc = wilson_matrix(N, U, m, &D);
  if (rc) return rc;
  double c = m + 2.0;
  eb->c = c;
  triplets te = {0}, to = {0};
  for (int y = 0; y < N && !rc; ++y)
    for (int x = 0; x < N && !rc; ++x) {
      int z = y * N + x, par = (x + y) & 1, hz = half_index(N, x, y);
      for (int s = 0; s < 2 && !rc; ++s) {
        int row = 2 * z + s;
        for (int p = D.rowptr[row]; p < D.rowptr[row + 1] && !rc; ++p) {
          int zc = D.col[p] / 2, sc = D.col[p] % 2;
          int xc = zc % N, yc = zc / N;
          int parc = (xc + yc) & 1, hc = half_index(N, xc, yc);
          if (parc == par) {
            /* diagonal blocks must be c * I (Sec. 3.2) */
            cplx expect = (zc == z && sc == s) ? c : 0.0;
            if (cabs(D.val[p] - expect) > 1e-14 * (1.0 + fabs(c))) rc = OR_ESTRUCT;
            continue;
          }
          if (par == 0)
            rc = trip_push(&te, 2 * hz + s, 2 * hc + sc, D.val[p] / c);
          else
            rc = trip_push(&to, 2 * hz + s, 2 * hc + sc, D.val[p] / c);
        }
      }
    }
  int nh = N * N / 2;
  if (!rc) rc = csr_from_triplets(2 * nh, 2 * nh, &te, &eb->Deo);
  if (!rc) rc = csr_from_triplets(2 * nh, 2 * nh, &to, &eb->Doe);
  trip_free(&te);
  trip_free(&to);
  csr_free(&D);
  return rc;
}

static void eo_free(eo_blocks *eb) {
  csr_free(&eb->Deo);
  csr_free(&eb->Doe);
}

static int dhat_matrix(int N, const cplx *U, double m, or_csr *Dh) {
  eo_blocks eb;
  int rc = eo_split(N, U, m, &eb);
  if (rc) return rc;
  or_csr prod;
  rc = csr_mul(&eb.Deo, &eb.Doe, &prod);
  if (!rc) {
    triplets t = {0};
    for (int i = 0; i < prod.nrow && !rc; ++i) {
      rc = trip_push(&t, i, i, 1.0);
      for (int p = prod.rowptr[i]; p < prod.rowptr[i + 1] && !rc; ++p)
        rc = trip_push(&t, i, prod.col[p], -prod.val[p]);
    }
    if (!rc) rc = csr_from_triplets(prod.nrow, prod.ncol, &t, Dh);
    trip_free(&t);
    csr_free(&prod);
  }
  eo_free(&eb);
  return rc;
}

int or_dhat_nnz(int N, const cplx *U, double m) {
  or_csr Dh;
  int rc = dhat_matrix(N, U, m, &Dh);
  if (rc) return rc;
  int nnz = Dh.nnz;
  csr_free(&Dh);
  return nnz;
}

int or_dhat_csr(int N, const cplx *U, double m, int *rowptr, int *col, cplx *val) {
  or_csr Dh;
  int rc = dhat_matrix(N, U, m, &Dh);
  if (rc) return rc;
  memcpy(rowptr, Dh.rowptr, sizeof(int) * ((size_t)Dh.nrow + 1));
  memcpy(col, Dh.col, sizeof(int) * (size_t)Dh.nnz);
  memcpy(val, Dh.val, sizeof(cplx) * (size_t)Dh.nnz);
  int nnz = Dh.nnz;
  csr_free(&Dh);
  return nnz;
}

/* Eq. (3.2) applied as two successive products, without forming Dhat. */
int or_dhat_apply(int N, const cplx *U, double m, const cplx *xe, cplx *ye) {
  eo_blocks eb;
  int rc = eo_split(N, U, m, &eb);
  if (rc) return rc;
  int n = eb.Doe.nrow;
  cplx *t = malloc(sizeof(cplx) * n);
  if (!t) { eo_free(&eb); return OR_ENOMEM; }
  csr_matvec(&eb.Doe, xe, t);
  csr_matvec(&eb.Deo, t, ye);
  for (int i = 0; i < n; ++i) ye[i] = xe[i] - ye[i];
  free(t);
  eo_free(&eb);
  return OR_OK;
}

/* Sec. 3.2, step 1 of the two-step solve with the 1/c scaling:
 * bhat = b'_e - (D_eo/c) b'_o, b' = b / c.  b is a full field [N][N][2]. */
int or_eo_reduce(int N, const cplx *U, double m, const cplx *b, cplx *bhat) {
  eo_blocks eb;
  int rc = eo_split(N, U, m, &eb);
  if (rc) return rc;
  int n = eb.Deo.nrow;
  cplx *be = malloc(sizeof(cplx) * n), *bo = malloc(sizeof(cplx) * n);
  if (!be || !bo) { free(be); free(bo); eo_free(&eb); return OR_ENOMEM; }
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x)
      for (int s = 0; s < 2; ++s) {
        cplx v = b[((size_t)y * N + x) * 2 + s] / eb.c;
        if (((x + y) & 1) == 0) be[2 * half_index(N, x, y) + s] = v;
        else bo[2 * half_index(N, x, y) + s] = v;
      }
  csr_matvec(&eb.Deo, bo, bhat);
  for (int i = 0; i < n; ++i) bhat[i] = be[i] - bhat[i];
  free(be); free(bo);
  eo_free(&eb);
  return OR_OK;
}

/* Sec. 3.2, step 2.  Reading: the printed "psi_o = psi_o - D_oe x_e" is
 * psi_o = b'_o - (D_oe/c) psi_e. */
int or_eo_reconstruct(int N, const cplx *U, double m, const cplx *b,
                      const cplx *xe, cplx *psi) {
  eo_blocks eb;
  int rc = eo_split(N, U, m, &eb);
  if (rc) return rc;
  int n = eb.Doe.nrow;
  cplx *t = malloc(sizeof(cplx) * n);
  if (!t) { eo_free(&eb); return OR_ENOMEM; }
  csr_matvec(&eb.Doe, xe, t);
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x)
      for (int s = 0; s < 2; ++s) {
        int h = half_index(N, x, y);
        size_t z = ((size_t)y * N + x) * 2 + s;
        if (((x + y) & 1) == 0) psi[z] = xe[2 * h + s];
        else psi[z] = b[z] / eb.c - t[2 * h + s];
      }
  free(t);
  eo_free(&eb);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Level geometry.  Level l is the even sublattice of an N_l x N_l torus;    */
/* site h <-> (x, y) with y = h / (N/2), x = 2 (h mod N/2) + (y mod 2).      */
/* Rotated coordinates a = (x+y)/2, b = (x-y)/2 make Dhat a 3x3 box stencil  */
/* (Sec. 3.2, Fig. 3.1 (b)); stencil offset d = 3 (da+1) + (db+1).           */
/* ------------------------------------------------------------------------ */
static void site_xy(int N, int h, int *x, int *y) {
  *y = h / (N / 2);
  *x = 2 * (h % (N / 2)) + (*y & 1);
}

static int wrap(int v, int N) { return ((v % N) + N) % N; }

static int site_of(int N, int x, int y) {
  x = wrap(x, N);
  y = wrap(y, N);
  return half_index(N, x, y);
}

int or_stencil_neighbour(int N, int h, int d) {
  int x, y;
  site_xy(N, h, &x, &y);
  int da = d / 3 - 1, db = d % 3 - 1;
  return site_of(N, x + da + db, y + da - db);
}

static int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }
static int posmod(int a, int b) { return ((a % b) + b) % b; }

/* Reading (Sec. 3.1: a colouring is "straightforward"): 16 colours
 * (a mod 4, b mod 4).  Same-colour sites are >= 4 apart in a and b, so the
 * 3x3 column supports of their variables are disjoint.  Needs N = 0 mod 8. */
int or_colour(int N, int h) {
  int x, y;
  site_xy(N, h, &x, &y);
  int a = (x + y) / 2, b = (x - y) / 2;
  return 4 * posmod(a, 4) + posmod(b, 4);
}

/* Reading of full coarsening (Sec. 3.2) with cell size B: coarse points are
 * a = 0 mod B, b = 0 mod B; each fine variable interpolates from the same
 * spin at the <= 4 corners of its B x B cell in (a, b).  For B = 2 these
 * corners are exactly the coarse neighbours in the graph of Dhat, Eq. (3.15).
 * corner k = ka + 2 kb; returns the number of existing corners and fills
 * the coarse site of each corner (-1 if absent). */
static int cell_corners(int N, int B, int h, int cs[4]) {
  int x, y;
  site_xy(N, h, &x, &y);
  int a = (x + y) / 2, b = (x - y) / 2;
  int a0 = B * floordiv(a, B), b0 = B * floordiv(b, B);
  int ra = a - a0, rb = b - b0;
  int Nc = N / B, cnt = 0;
  for (int k = 0; k < 4; ++k) {
    int ka = k & 1, kb = k >> 1;
    if ((ka && !ra) || (kb && !rb)) { cs[k] = -1; continue; }
    int ac = a0 + ka * B, bc = b0 + kb * B;
    int xc = wrap(ac + bc, N), yc = wrap(ac - bc, N);
    cs[k] = site_of(Nc, xc / B, yc / B);
    cnt++;
  }
  return cnt;
}

/* fine site that carries coarse site hc (the C point) */
static int c_point(int Nc, int B, int hc) {
  int xc, yc;
  site_xy(Nc, hc, &xc, &yc);
  return site_of(Nc * B, xc * B, yc * B);
}

/* ------------------------------------------------------------------------ */
/* Hierarchy containers.                                                    */
/* ------------------------------------------------------------------------ */
static int n_sites(int N) { return N * N / 2; }

static int build_P(int Nf, int B, const cplx *Pw, or_csr *P) {
  int nf = n_sites(Nf), nc = n_sites(Nf / B);
  triplets t = {0};
  int rc = OR_OK;
  for (int h = 0; h < nf && !rc; ++h) {
    int cs[4];
    cell_corners(Nf, B, h, cs);
    for (int s = 0; s < 2 && !rc; ++s)
      for (int k = 0; k < 4 && !rc; ++k)
        if (cs[k] >= 0) rc = trip_push(&t, 2 * h + s, 2 * cs[k] + s, Pw[((size_t)h * 2 + s) * 4 + k]);
  }
  if (!rc) rc = csr_from_triplets(2 * nf, 2 * nc, &t, P);
  trip_free(&t);
  return rc;
}

static int stencil_to_csr(int N, const cplx *As, or_csr *A) {
  int n = n_sites(N);
  triplets t = {0};
  int rc = OR_OK;
  for (int h = 0; h < n && !rc; ++h)
    for (int d = 0; d < 9 && !rc; ++d) {
      int j = or_stencil_neighbour(N, h, d);
      for (int s = 0; s < 2 && !rc; ++s)
        for (int u = 0; u < 2 && !rc; ++u)
          rc = trip_push(&t, 2 * h + s, 2 * j + u, As[(((size_t)h * 9 + d) * 2 + s) * 2 + u]);
    }
  if (!rc) rc = csr_from_triplets(2 * n, 2 * n, &t, A);
  trip_free(&t);
  return rc;
}

static int csr_to_stencil(int N, const or_csr *A, cplx *As) {
  int n = n_sites(N);
  memset(As, 0, sizeof(cplx) * (size_t)n * 36);
  for (int row = 0; row < A->nrow; ++row) {
    int h = row / 2, s = row % 2;
    for (int p = A->rowptr[row]; p < A->rowptr[row + 1]; ++p) {
      int j = A->col[p] / 2, u = A->col[p] % 2, found = 0;
      for (int d = 0; d < 9; ++d)
        if (or_stencil_neighbour(N, h, d) == j) {
          As[(((size_t)h * 9 + d) * 2 + s) * 2 + u] += A->val[p];
          found = 1;
          break;
        }
      if (!found && A->val[p] != 0) return OR_ESTRUCT;
    }
  }
  return OR_OK;
}

/* textbook LU with partial pivoting (row major), in place */
static int dense_lu(int n, cplx *a, int *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = cabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (cabs(a[(size_t)i * n + k]) > best) { best = cabs(a[(size_t)i * n + k]); p = i; }
    if (best == 0.0) return OR_ESTRUCT;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        cplx t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)p * n + j];
        a[(size_t)p * n + j] = t;
      }
    for (int i = k + 1; i < n; ++i) {
      cplx l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return OR_OK;
}

static void lu_solve(int n, const cplx *lu, const int *piv, const cplx *b, cplx *x) {
  if (x != b) memcpy(x, b, sizeof(cplx) * n);
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) { cplx t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) x[i] -= lu[(size_t)i * n + j] * x[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) x[i] -= lu[(size_t)i * n + j] * x[j];
    x[i] /= lu[(size_t)i * n + i];
  }
}

int or_dense_lu_solve(int n, const cplx *A, const cplx *b, cplx *x) {
  cplx *a = malloc(sizeof(cplx) * (size_t)n * n);
  int *piv = malloc(sizeof(int) * n);
  if (!a || !piv) { free(a); free(piv); return OR_ENOMEM; }
  memcpy(a, A, sizeof(cplx) * (size_t)n * n);
  int rc = dense_lu(n, a, piv);
  if (!rc) lu_solve(n, a, piv, b, x);
  free(a); free(piv);
  return rc;
}

static int hier_coarsest_lu(or_hier *h) {
  int l = h->L - 1;
  int n = h->A[l].nrow;
  free(h->lu);
  free(h->piv);
  h->lu = malloc(sizeof(cplx) * (size_t)n * n);
  h->piv = malloc(sizeof(int) * n);
  if (!h->lu || !h->piv) return OR_ENOMEM;
  h->nc = n;
  or_csr_dense(&h->A[l], h->lu);
  return dense_lu(n, h->lu, h->piv);
}

void or_hier_free(or_hier *h) {
  if (!h) return;
  for (int l = 0; l < OR_MAXLEV; ++l) {
    csr_free(&h->A[l]);
    csr_free(&h->AT[l]);
    csr_free(&h->P[l]);
    csr_free(&h->PH[l]);
    csr_free(&h->T[l]);
  }
  free(h->lu);
  free(h->piv);
  free(h);
}

int or_hier_levels(const or_hier *h, int *Nl, int *Bl) {
  for (int l = 0; l < h->L; ++l) { Nl[l] = h->N[l]; Bl[l] = h->B[l]; }
  return h->L;
}

static int check_levels(int N, int L, const int *Nl, const int *Bl) {
  if (L < 2 || L > OR_MAXLEV || Nl[0] != N) return OR_EINVAL;
  for (int l = 0; l + 1 < L; ++l) {
    if (Bl[l] < 2 || Nl[l] % Bl[l] || (Nl[l] / 2) % Bl[l]) return OR_EINVAL;
    if (Nl[l + 1] != Nl[l] / Bl[l]) return OR_EINVAL;
    if (Nl[l] % 8) return OR_EINVAL;
  }
  return Nl[L - 1] >= 4 ? OR_OK : OR_EINVAL;
}

/* Build a hierarchy from interpolation weights Pw[l] ([n_l][2][4]) and
 * coarse stencils As[l] ([n_l][9][2][2], l >= 1).  Level 0 is Dhat. */
or_hier *or_hier_import(int N, const cplx *U, double m, int L, const int *Nl,
                        const int *Bl, const cplx *const *Pw,
                        const cplx *const *As) {
  if (check_levels(N, L, Nl, Bl)) return NULL;
  or_hier *h = calloc(1, sizeof(or_hier));
  if (!h) return NULL;
  h->L = L;
  h->Nfine = N;
  h->m = m;
  int rc = OR_OK;
  for (int l = 0; l < L; ++l) { h->N[l] = Nl[l]; h->B[l] = (l + 1 < L) ? Bl[l] : 0; }
  rc = dhat_matrix(N, U, m, &h->A[0]);
  for (int l = 1; l < L && !rc; ++l) rc = stencil_to_csr(Nl[l], As[l], &h->A[l]);
  for (int l = 0; l < L && !rc; ++l) rc = csr_transpose(&h->A[l], 0, &h->AT[l]);
  for (int l = 0; l + 1 < L && !rc; ++l) {
    rc = build_P(Nl[l], Bl[l], Pw[l], &h->P[l]);
    if (!rc) rc = csr_transpose(&h->P[l], 1, &h->PH[l]);
  }
  if (!rc) rc = hier_coarsest_lu(h);
  if (rc) { or_hier_free(h); return NULL; }
  return h;
}

int or_hier_export(const or_hier *h, cplx *const *Pw, cplx *const *As) {
  for (int l = 0; l + 1 < h->L; ++l) {
    int nf = n_sites(h->N[l]);
    memset(Pw[l], 0, sizeof(cplx) * (size_t)nf * 8);
    for (int row = 0; row < h->P[l].nrow; ++row) {
      int hf = row / 2, s = row % 2, cs[4];
      cell_corners(h->N[l], h->B[l], hf, cs);
      for (int p = h->P[l].rowptr[row]; p < h->P[l].rowptr[row + 1]; ++p) {
        int j = h->P[l].col[p] / 2, found = 0;
        for (int k = 0; k < 4; ++k)
          if (cs[k] == j) { Pw[l][((size_t)hf * 2 + s) * 4 + k] = h->P[l].val[p]; found = 1; break; }
        if (!found) return OR_ESTRUCT;
      }
    }
  }
  for (int l = 1; l < h->L; ++l) {
    int rc = csr_to_stencil(h->N[l], &h->A[l], As[l]);
    if (rc) return rc;
  }
  return OR_OK;
}

int or_hier_level_dense(const or_hier *h, int l, int which, cplx *dense) {
  if (l < 0 || l >= h->L) return OR_EINVAL;
  const or_csr *M = which == 0 ? &h->A[l] : which == 1 ? &h->P[l] : &h->T[l];
  if (!M->rowptr) return OR_EINVAL;
  return or_csr_dense(M, dense);
}

/* ------------------------------------------------------------------------ */
/* Solve-phase steps.                                                       */
/* ------------------------------------------------------------------------ */
int or_level_apply(const or_hier *h, int l, const cplx *x, cplx *y) {
  if (l < 0 || l >= h->L) return OR_EINVAL;
  csr_matvec(&h->A[l], x, y);
  return OR_OK;
}

/* Sec. 3.1: Kaczmarz relaxation in the normal-equation (column) form.  For
 * variable i: s_i = <r, A e_i> / ||A e_i||^2 with <x, y> = y^H x, then
 * x_i += omega s_i and r -= omega s_i A e_i (the exact line minimiser of
 * ||r||; the printed "+" sign in the residual update is read as "-").
 * order LEX: i = 0 .. 2n-1 (site-major, spin 0 then 1, the forward sweep).
 * order COLOUR: colours 0..15 in turn; within a colour the sites in
 * increasing index (or in the order perm[] when given), spin 0 then 1. */
static void kaczmarz_update(const or_csr *AT, int i, cplx *x, cplx *r, double omega) {
  cplx num = 0;
  double den = 0;
  for (int p = AT->rowptr[i]; p < AT->rowptr[i + 1]; ++p) {
    num += conj(AT->val[p]) * r[AT->col[p]];
    den += creal(AT->val[p]) * creal(AT->val[p]) + cimag(AT->val[p]) * cimag(AT->val[p]);
  }
  if (den == 0.0) return;
  cplx s = omega * num / den;
  x[i] += s;
  for (int p = AT->rowptr[i]; p < AT->rowptr[i + 1]; ++p) r[AT->col[p]] -= s * AT->val[p];
}

/* Tile-coloured ordering (a reading of Sec. 3.1's parallel ordering that
 * keeps each tile's work local): the (a, b) plane is cut into T x T tiles,
 * tile (ta, tb) = (a / T, b / T) of the fundamental domain a in [0, N),
 * b in [0, N/2), with tile colour (ta mod 2) + 2 (tb mod 2).  The sweep takes
 * tile colours 0..3 in turn; inside a tile it takes the 16 site colours
 * 4 (a mod 4) + (b mod 4) along the 4 x 4 colour grid row by row, even rows
 * left to right and odd rows right to left (serpentine: 0 1 2 3 7 6 5 4
 * 8 9 10 11 15 14 13 12), sites of a colour in increasing (a, b), spin 0
 * then 1.  Any order of the colours is a multicolour ordering; in this one
 * the sites of consecutive colours are neighbours in a row or a column.  Variables of a
 * site touch only its 3x3 (a, b) box, so tiles of one colour (one tile
 * apart) are independent.  T = 8 when N >= 64 (then 4T divides N, which
 * keeps the tile colouring consistent across the seam b = N/2 ~ 0);
 * smaller grids use the plain 16-colour order. */
int or_tile_size(int N) { return (N >= 64 && N % 32 == 0) ? 8 : 0; }

static void tile_sweep(const or_csr *AT, int N, cplx *x, cplx *r, double omega) {
  int T = or_tile_size(N);
  for (int tc = 0; tc < 4; ++tc)
#pragma omp parallel for collapse(2) schedule(static)
    for (int ta = 0; ta < N / T; ++ta)
      for (int tb = 0; tb < N / (2 * T); ++tb) {
        if ((ta & 1) + 2 * (tb & 1) != tc) continue;
        for (int s = 0; s < 16; ++s) {
          int row = s / 4, col = (row % 2) ? 3 - s % 4 : s % 4, c = 4 * row + col;
          for (int i = 0; i < T; ++i)
            for (int j = 0; j < T; ++j) {
              int a = ta * T + i, b = tb * T + j;
              if (4 * (a % 4) + (b % 4) != c) continue;
              int site = site_of(N, a + b, a - b);
              kaczmarz_update(AT, 2 * site, x, r, omega);
              kaczmarz_update(AT, 2 * site + 1, x, r, omega);
            }
        }
      }
}

int or_kaczmarz(const or_hier *h, int l, cplx *x, cplx *r, int order, int sweeps,
                double omega, const int *perm) {
  if (l < 0 || l >= h->L) return OR_EINVAL;
  const or_csr *AT = &h->AT[l];
  int N = h->N[l], n = AT->nrow / 2;
  if (order != OR_ORDER_LEX && N % 8) return OR_EINVAL;
  if (order == OR_ORDER_TILE && !or_tile_size(N)) order = OR_ORDER_COLOUR;
  for (int sw = 0; sw < sweeps; ++sw) {
    if (order == OR_ORDER_TILE) {
      tile_sweep(AT, N, x, r, omega);
    } else if (order == OR_ORDER_LEX) {
      for (int i = 0; i < 2 * n; ++i) kaczmarz_update(AT, i, x, r, omega);
    } else {
      for (int k = 0; k < 16; ++k)
#pragma omp parallel for schedule(static)
        for (int q = 0; q < n; ++q) {
          int site = perm ? perm[q] : q;
          if (or_colour(N, site) != k) continue;
          kaczmarz_update(AT, 2 * site, x, r, omega);
          kaczmarz_update(AT, 2 * site + 1, x, r, omega);
        }
    }
  }
  return OR_OK;
}

/* Sec. 1 / Sec. 3.5: Galerkin restriction is P^H */
int or_restrict(const or_hier *h, int l, const cplx *r, cplx *fc) {
  if (l < 0 || l + 1 >= h->L) return OR_EINVAL;
  csr_matvec(&h->PH[l], r, fc);
  return OR_OK;
}

int or_prolong(const or_hier *h, int l, const cplx *e, cplx *x) {
  if (l < 0 || l + 1 >= h->L) return OR_EINVAL;
  int n = h->P[l].nrow;
  cplx *t = malloc(sizeof(cplx) * n);
  if (!t) return OR_ENOMEM;
  csr_matvec(&h->P[l], e, t);
  for (int i = 0; i < n; ++i) x[i] += t[i];
  free(t);
  return OR_OK;
}

/* Sec. 4: the coarsest system is solved directly (dense LU). */
int or_coarsest_solve(const or_hier *h, const cplx *f, cplx *x) {
  lu_solve(h->nc, h->lu, h->piv, f, x);
  return OR_OK;
}

/* Sec. 1: two-grid correction E = (I - P A_c^{-1} P^H A)(I - M A) with pre-
 * and post-smoothing, applied recursively; gamma = 1 is a V-cycle, gamma = 2
 * a W-cycle (Sec. 4).  Starts from x = 0 and returns x ~ A_l^{-1} f. */
int or_cycle(const or_hier *h, int l, const cplx *f, cplx *x, int nu1, int nu2,
             int gamma, int order) {
  if (l == h->L - 1) return or_coarsest_solve(h, f, x);
  int n = h->A[l].nrow, nc = h->A[l + 1].nrow;
  cplx *r = malloc(sizeof(cplx) * n);
  cplx *fc = malloc(sizeof(cplx) * nc), *ec = calloc(nc, sizeof(cplx));
  cplx *rc_ = malloc(sizeof(cplx) * nc), *dc = malloc(sizeof(cplx) * nc);
  if (!r || !fc || !ec || !rc_ || !dc) { free(r); free(fc); free(ec); free(rc_); free(dc); return OR_ENOMEM; }
  int ord = (h->N[l] % 8) ? OR_ORDER_LEX : order;
  for (int i = 0; i < n; ++i) { x[i] = 0; r[i] = f[i]; }
  int rc = or_kaczmarz(h, l, x, r, ord, nu1, 1.0, NULL);
  if (!rc) rc = or_restrict(h, l, r, fc);
  for (int g = 0; g < gamma && !rc; ++g) {
    if (g == 0) {
      rc = or_cycle(h, l + 1, fc, ec, nu1, nu2, gamma, order);
    } else {
      csr_matvec(&h->A[l + 1], ec, rc_);
      for (int i = 0; i < nc; ++i) rc_[i] = fc[i] - rc_[i];
      rc = or_cycle(h, l + 1, rc_, dc, nu1, nu2, gamma, order);
      for (int i = 0; i < nc && !rc; ++i) ec[i] += dc[i];
    }
  }
  if (!rc) rc = or_prolong(h, l, ec, x);
  if (!rc) {
    csr_matvec(&h->A[l], x, r);
    for (int i = 0; i < n; ++i) r[i] = f[i] - r[i];
    rc = or_kaczmarz(h, l, x, r, ord, nu2, 1.0, NULL);
  }
  free(r); free(fc); free(ec); free(rc_); free(dc);
  return rc;
}

static double vnorm(int n, const cplx *v) {
  double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
  return sqrt(s);
}

static cplx vdot(int n, const cplx *a, const cplx *b) { /* a^H b */
  double sr = 0, si = 0;
#pragma omp parallel for reduction(+ : sr, si) schedule(static)
  for (int i = 0; i < n; ++i) {
    cplx t = conj(a[i]) * b[i];
    sr += creal(t);
    si += cimag(t);
  }
  return CMPLX(sr, si);
}

/* Flexible GMRES(m) (Saad 1993) with right preconditioning z_j = M(v_j),
 * classical Gram-Schmidt (gs_passes = 1) or classical Gram-Schmidt with one
 * reorthogonalisation (gs_passes = 2), and Givens rotations.  Sec. 4 uses
 * GMRES(32) preconditioned by a W(4,4) cycle; any cycle is allowed here.
 * At each restart the true residual is recomputed.  precond = 0: identity
 * (plain GMRES); 1, 2, 3: the cycle with the 16-colour, tile-coloured or
 * lexicographic Kaczmarz ordering.  Returns 0 converged, 1 not. */
int or_fgmres(const or_hier *h, const cplx *b, cplx *x, double tol, int mrestart,
              int max_restarts, int nu1, int nu2, int gamma, int precond, int gs_passes,
              int *iters_out, int *restarts_out, double *relres_out) {
  int n = h->A[0].nrow, m = mrestart;
  if (gs_passes < 1 || gs_passes > 2 || precond < 0 || precond > 3 || m < 1 || m > 64) return OR_EINVAL;
  const int cyc_order[4] = {0, OR_ORDER_COLOUR, OR_ORDER_TILE, OR_ORDER_LEX};
  cplx *V = malloc(sizeof(cplx) * (size_t)n * (m + 1));
  cplx *Z = malloc(sizeof(cplx) * (size_t)n * m);
  cplx *w = malloc(sizeof(cplx) * n), *r = malloc(sizeof(cplx) * n);
  cplx *H = calloc((size_t)(m + 1) * m, sizeof(cplx));
  cplx *g = calloc(m + 1, sizeof(cplx)), *cs = malloc(sizeof(cplx) * m);
  double *cc = malloc(sizeof(double) * m);
  cplx *hcol = malloc(sizeof(cplx) * (m + 1)), *y = malloc(sizeof(cplx) * m);
  if (!V || !Z || !w || !r || !H || !g || !cs || !cc || !hcol || !y) {
    free(V); free(Z); free(w); free(r); free(H); free(g); free(cs); free(cc); free(hcol); free(y);
    return OR_ENOMEM;
  }
  double bnorm = vnorm(n, b);
  if (bnorm == 0) bnorm = 1;
  int iters = 0, restarts = 0, status = 1, rc = OR_OK;
  double relres = 0;
  for (;;) {
    csr_matvec(&h->A[0], x, r);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double beta = vnorm(n, r);
    relres = beta / bnorm;
    if (relres <= tol) { status = 0; break; }
    if (restarts >= max_restarts) break;
    for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0;
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m; ++j) {
      cplx *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
      if (precond) rc = or_cycle(h, 0, vj, zj, nu1, nu2, gamma, cyc_order[precond]);
      else memcpy(zj, vj, sizeof(cplx) * n);
      if (rc) break;
      csr_matvec(&h->A[0], zj, w);
      for (int k = 0; k <= j; ++k) hcol[k] = 0;
      for (int pass = 0; pass < gs_passes; ++pass) {
        cplx hp[64];
        for (int k = 0; k <= j; ++k) hp[k] = vdot(n, V + (size_t)k * n, w);
        for (int k = 0; k <= j; ++k) {
          const cplx *vk = V + (size_t)k * n;
#pragma omp parallel for schedule(static)
          for (int i = 0; i < n; ++i) w[i] -= hp[k] * vk[i];
          hcol[k] += hp[k];
        }
      }
      double hn = vnorm(n, w);
      hcol[j + 1] = hn;
      if (hn > 0)
        for (int i = 0; i < n; ++i) V[(size_t)(j + 1) * n + i] = w[i] / hn;
      /* previous rotations */
      for (int k = 0; k < j; ++k) {
        cplx t = cc[k] * hcol[k] + cs[k] * hcol[k + 1];
        hcol[k + 1] = -conj(cs[k]) * hcol[k] + cc[k] * hcol[k + 1];
        hcol[k] = t;
      }
      /* new rotation zeroing hcol[j+1] */
      double a = cabs(hcol[j]), bb = cabs(hcol[j + 1]);
      double den = sqrt(a * a + bb * bb);
      if (den == 0) { cc[j] = 1; cs[j] = 0; }
      else if (a == 0) { cc[j] = 0; cs[j] = conj(hcol[j + 1]) / bb; }
      else {
        cc[j] = a / den;
        cs[j] = (hcol[j] / a) * conj(hcol[j + 1]) / den;
      }
      hcol[j] = cc[j] * hcol[j] + cs[j] * hcol[j + 1];
      hcol[j + 1] = 0;
      g[j + 1] = -conj(cs[j]) * g[j];
      g[j] = cc[j] * g[j];
      for (int k = 0; k <= j; ++k) H[(size_t)k * m + j] = hcol[k];
      iters++;
      jend = j + 1;
      if (cabs(g[j + 1]) / bnorm <= tol || hn == 0) break;
    }
    if (rc) break;
    for (int i = jend - 1; i >= 0; --i) {
      cplx s = g[i];
      for (int k = i + 1; k < jend; ++k) s -= H[(size_t)i * m + k] * y[k];
      y[i] = s / H[(size_t)i * m + i];
    }
    for (int k = 0; k < jend; ++k)
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) x[i] += y[k] * Z[(size_t)k * n + i];
    restarts++;
  }
  if (iters_out) *iters_out = iters;
  if (restarts_out) *restarts_out = restarts;
  if (relres_out) *relres_out = relres;
  free(V); free(Z); free(w); free(r); free(H); free(g); free(cs); free(cc); free(hcol); free(y);
  return rc ? rc : status;
}

/* Sec. 4, convergence estimate of the stand-alone solver: the cycle used as
 * a stationary iteration x <- x + M(f - A_0 x) on A_0 x = 0, so the iterate
 * is the error, e^nu = (I - M A_0) e^{nu-1} with e^0 = x0.  rho is
 * |e^nu| / |e^{nu-1}| at the first nu with |e^nu| <= tol |e^0|, or at
 * nu = maxit.  hist (optional, maxit + 1 entries): |e^k| for k <= nu.
 * Reading: a divergent iteration (the paper's definition presumes
 * convergence) stops when the error norm overflows; rho is then the ratio of
 * the last two finite norms and nu the last finite iteration.
 * Returns 0 when the tolerance was met, 1 otherwise. */
int or_rho(const or_hier *h, const cplx *x0, double tol, int maxit, int nu1, int nu2,
           int gamma, int order, double *rho_out, int *iters_out, double *hist) {
  int n = h->A[0].nrow;
  cplx *e = malloc(sizeof(cplx) * n), *w = malloc(sizeof(cplx) * n);
  cplx *c = malloc(sizeof(cplx) * n);
  if (!e || !w || !c) { free(e); free(w); free(c); return OR_ENOMEM; }
  for (int i = 0; i < n; ++i) e[i] = x0[i];
  double n0 = vnorm(n, e), prev = n0, rho = 0;
  if (hist) hist[0] = n0;
  int nu = 0, rc = 0, met = 0;
  while (nu < maxit && !rc) {
    csr_matvec(&h->A[0], e, w);                 /* residual of A_0 x = 0 is -A_0 e */
    rc = or_cycle(h, 0, w, c, nu1, nu2, gamma, order);
    if (rc) break;
    for (int i = 0; i < n; ++i) e[i] -= c[i];   /* x + M(-A_0 x) = x - M(A_0 x) */
    double cur = vnorm(n, e);
    if (!isfinite(cur)) break;                  /* diverged past overflow: keep the last ratio */
    ++nu;
    if (hist) hist[nu] = cur;
    rho = prev > 0 ? cur / prev : 0;
    prev = cur;
    if (cur <= tol * n0) { met = 1; break; }
  }
  free(e); free(w); free(c);
  if (rc) return rc;
  *rho_out = rho;
  *iters_out = nu;
  return met ? 0 : 1;
}

/* Sec. 4: D psi = b through the reduced system Dhat psi_e = bhat. */
int or_solve(int N, const cplx *U, double m, const or_hier *h, const cplx *b,
             cplx *psi, double tol, int mrestart, int max_restarts, int nu1,
             int nu2, int gamma, int order, int gs_passes, int *iters_out, double *relres_out) {
  int n = n_sites(N) * 2;
  cplx *bh = malloc(sizeof(cplx) * n), *xe = calloc(n, sizeof(cplx));
  if (!bh || !xe) { free(bh); free(xe); return OR_ENOMEM; }
  int rc = or_eo_reduce(N, U, m, b, bh);
  int st = 1;
  int precond = order == OR_ORDER_TILE ? 2 : order == OR_ORDER_LEX ? 3 : 1;
  if (!rc) st = or_fgmres(h, bh, xe, tol, mrestart, max_restarts, nu1, nu2, gamma,
                          precond, gs_passes, iters_out, NULL, relres_out);
  if (!rc && st >= 0) rc = or_eo_reconstruct(N, U, m, b, xe, psi);
  free(bh); free(xe);
  return rc ? rc : st;
}

/* ------------------------------------------------------------------------ */
/* Setup building blocks.                                                   */
/* ------------------------------------------------------------------------ */

/* cyclic Jacobi for a Hermitian matrix (row major, overwritten); eigen-
 * vectors in the columns of Q.  Textbook two-sided rotations. */
static void herm_jacobi(int n, cplx *A, cplx *Q, double *lam) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Q[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0;
  for (size_t k = 0; k < (size_t)n * n; ++k) fro += creal(A[k] * conj(A[k]));
  fro = sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += creal(A[(size_t)p * n + q] * conj(A[(size_t)p * n + q]));
    if (sqrt(off) <= 1e-16 * fro || fro == 0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        cplx apq = A[(size_t)p * n + q];
        double ab = cabs(apq);
        if (ab == 0.0) continue;
        cplx e = apq / ab;
        double app = creal(A[(size_t)p * n + p]), aqq = creal(A[(size_t)q * n + q]);
        double tau = (aqq - app) / (2.0 * ab);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* G = I with G_pp = G_qq = c, G_pq = s e, G_qp = -s conj(e); A <- G^H A G */
        for (int k = 0; k < n; ++k) { /* columns */
          cplx akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * conj(e) * akq;
          A[(size_t)k * n + q] = s * e * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* rows */
          cplx apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * e * aqk;
          A[(size_t)q * n + k] = s * conj(e) * apk + c * aqk;
        }
        A[(size_t)p * n + q] = 0;
        A[(size_t)q * n + p] = 0;
        A[(size_t)p * n + p] = creal(A[(size_t)p * n + p]);
        A[(size_t)q * n + q] = creal(A[(size_t)q * n + q]);
        for (int k = 0; k < n; ++k) {
          cplx qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - s * conj(e) * qkq;
          Q[(size_t)k * n + q] = s * e * qkp + c * qkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = creal(A[(size_t)i * n + i]);
}

/* Sec. 3.3, Eq. (3.4): for every fine variable i (site h, spin s) that is not
 * a C point, minimise sum_k w_k |v_i^k - sum_{j in C_i} p_ij v_j^k|^2 over
 * the same-spin cell corners C_i.  Normal equations M p = g with
 * M_jl = sum_k w_k conj(v_j^k) v_l^k, g_j = sum_k w_k conj(v_j^k) v_i^k,
 * solved with an eigen-pseudoinverse (eigenvalues below 1e-12 trace(M) are
 * dropped).  C points get the identity row.  V is [k][2 n_f] (test vectors
 * on the fine level); Pw is [n_f][2][4]. */
int or_ls_fit(int Nf, int B, int k, const cplx *V, const double *w, cplx *Pw) {
  int nf = n_sites(Nf);
  size_t stride = (size_t)2 * nf;
  for (int h = 0; h < nf; ++h) {
    int cs[4];
    int cnt = cell_corners(Nf, B, h, cs);
    int x, y;
    site_xy(Nf, h, &x, &y);
    /* coarse site index -> fine C-point index */
    int cf[4];
    for (int q = 0; q < 4; ++q) cf[q] = cs[q] >= 0 ? c_point(Nf / B, B, cs[q]) : -1;
    for (int s = 0; s < 2; ++s) {
      cplx *pw = Pw + ((size_t)h * 2 + s) * 4;
      for (int q = 0; q < 4; ++q) pw[q] = 0;
      if (cnt == 1) { pw[0] = 1.0; continue; } /* C point */
      int idx[4], nc = 0;
      for (int q = 0; q < 4; ++q) if (cs[q] >= 0) idx[nc++] = q;
      cplx M[16], g[4], Q[16];
      double mu[4];
      for (int a = 0; a < nc; ++a) {
        g[a] = 0;
        for (int b = 0; b < nc; ++b) M[a * nc + b] = 0;
      }
      for (int kk = 0; kk < k; ++kk) {
        const cplx *v = V + kk * stride;
        cplx vi = v[2 * h + s];
        for (int a = 0; a < nc; ++a) {
          cplx va = v[2 * cf[idx[a]] + s];
          g[a] += w[kk] * conj(va) * vi;
          for (int b = 0; b < nc; ++b) M[a * nc + b] += w[kk] * conj(va) * v[2 * cf[idx[b]] + s];
        }
      }
      double tr = 0;
      for (int a = 0; a < nc; ++a) tr += creal(M[a * nc + a]);
      herm_jacobi(nc, M, Q, mu);
      cplx p[4] = {0, 0, 0, 0};
      for (int e = 0; e < nc; ++e) {
        if (mu[e] <= 1e-12 * tr) continue;
        cplx qg = 0;
        for (int a = 0; a < nc; ++a) qg += conj(Q[a * nc + e]) * g[a];
        for (int a = 0; a < nc; ++a) p[a] += Q[a * nc + e] * qg / mu[e];
      }
      for (int a = 0; a < nc; ++a) pw[idx[a]] = p[a];
    }
  }
  return OR_OK;
}

/* Hermitian generalised eigenproblem Z v = lam T v (T Hermitian positive
 * definite): T = C C^H (Cholesky), C^-1 Z C^-H = Y Lam Y^H, V = C^-H Y, so
 * V^H T V = I.  Eigenvalues ascending in lam; V column major per vector:
 * V[k * n + i] is entry i of eigenvector k.  (Sec. 3.4, Thm. 3.1 (i).) */
int or_gen_eig(int n, const cplx *Z, const cplx *T, double *lam, cplx *V) {
  cplx *C = calloc((size_t)n * n, sizeof(cplx));
  cplx *M = malloc(sizeof(cplx) * (size_t)n * n), *Q = malloc(sizeof(cplx) * (size_t)n * n);
  cplx *W = malloc(sizeof(cplx) * (size_t)n * n);
  double *mu = malloc(sizeof(double) * n);
  int *ord = malloc(sizeof(int) * n);
  if (!C || !M || !Q || !W || !mu || !ord) { free(C); free(M); free(Q); free(W); free(mu); free(ord); return OR_ENOMEM; }
  int rc = OR_OK;
  for (int j = 0; j < n && !rc; ++j) { /* lower Cholesky T = C C^H */
    double d = creal(T[(size_t)j * n + j]);
    for (int k = 0; k < j; ++k) d -= creal(C[(size_t)j * n + k] * conj(C[(size_t)j * n + k]));
    if (d <= 0) { rc = OR_ESTRUCT; break; }
    C[(size_t)j * n + j] = sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      cplx s = T[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= C[(size_t)i * n + k] * conj(C[(size_t)j * n + k]);
      C[(size_t)i * n + j] = s / C[(size_t)j * n + j];
    }
  }
  if (!rc) {
    /* W = C^-1 Z (forward substitution per column) */
    for (int col = 0; col < n; ++col)
      for (int i = 0; i < n; ++i) {
        cplx s = Z[(size_t)i * n + col];
        for (int k = 0; k < i; ++k) s -= C[(size_t)i * n + k] * W[(size_t)k * n + col];
        W[(size_t)i * n + col] = s / C[(size_t)i * n + i];
      }
    /* M = W C^-H, i.e. M^H = C^-1 W^H: forward substitution on rows of W */
    for (int row = 0; row < n; ++row)
      for (int i = 0; i < n; ++i) {
        cplx s = conj(W[(size_t)row * n + i]);
        for (int k = 0; k < i; ++k) s -= C[(size_t)i * n + k] * conj(M[(size_t)row * n + k]);
        M[(size_t)row * n + i] = conj(s / C[(size_t)i * n + i]);
      }
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) { /* exact Hermitian part */
        cplx a = 0.5 * (M[(size_t)i * n + j] + conj(M[(size_t)j * n + i]));
        M[(size_t)i * n + j] = a;
        M[(size_t)j * n + i] = conj(a);
      }
    for (int i = 0; i < n; ++i) M[(size_t)i * n + i] = creal(M[(size_t)i * n + i]);
    herm_jacobi(n, M, Q, mu);
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 1; i < n; ++i) { /* sort ascending */
      int t = ord[i], j = i - 1;
      while (j >= 0 && mu[ord[j]] > mu[t]) { ord[j + 1] = ord[j]; j--; }
      ord[j + 1] = t;
    }
    for (int e = 0; e < n; ++e) {
      lam[e] = mu[ord[e]];
      /* back substitution C^H v = y */
      for (int i = n - 1; i >= 0; --i) {
        cplx s = Q[(size_t)i * n + ord[e]];
        for (int k = i + 1; k < n; ++k) s -= conj(C[(size_t)k * n + i]) * V[(size_t)e * n + k];
        V[(size_t)e * n + i] = s / conj(C[(size_t)i * n + i]);
      }
    }
  }
  free(C); free(M); free(Q); free(W); free(mu); free(ord);
  return rc;
}

/* Reading: Galerkin products are made exactly gamma_5-Hermitian (resp.
 * Hermitian for T) by averaging an entry with its mirror, which removes
 * rounding only (Sec. 3.5: the coarse operators satisfy the
 * gamma_5-symmetry). sign = 1: A = Gamma5 A^H Gamma5, sign = 0: T = T^H. */
static int csr_symmetrise(or_csr *A, int g5) {
  or_csr AH;
  int rc = csr_transpose(A, 1, &AH);
  if (rc) return rc;
  triplets t = {0};
  for (int i = 0; i < A->nrow && !rc; ++i) {
    for (int p = A->rowptr[i]; p < A->rowptr[i + 1] && !rc; ++p)
      rc = trip_push(&t, i, A->col[p], 0.5 * A->val[p]);
    for (int p = AH.rowptr[i]; p < AH.rowptr[i + 1] && !rc; ++p) {
      int j = AH.col[p];
      double sg = (g5 && ((i & 1) != (j & 1))) ? -1.0 : 1.0;
      rc = trip_push(&t, i, j, 0.5 * sg * AH.val[p]);
    }
  }
  or_csr S;
  if (!rc) rc = csr_from_triplets(A->nrow, A->ncol, &t, &S);
  trip_free(&t);
  csr_free(&AH);
  if (rc) return rc;
  csr_free(A);
  *A = S;
  return OR_OK;
}

/* Sec. 3.5: D_{l+1} = P^H D_l P (and T_{l+1} = P^H T_l P when T_l is held) */
static int galerkin_level(or_hier *h, int l) {
  or_csr AP, Ac;
  int rc = csr_mul(&h->A[l], &h->P[l], &AP);
  if (rc) return rc;
  rc = csr_mul(&h->PH[l], &AP, &Ac);
  csr_free(&AP);
  if (rc) return rc;
  rc = csr_symmetrise(&Ac, 1);
  if (rc) { csr_free(&Ac); return rc; }
  csr_free(&h->A[l + 1]);
  csr_free(&h->AT[l + 1]);
  h->A[l + 1] = Ac;
  rc = csr_transpose(&h->A[l + 1], 0, &h->AT[l + 1]);
  if (rc) return rc;
  if (h->nT) {
    or_csr TP, Tc;
    if (l == 0) rc = csr_mul(&h->PH[0], &h->P[0], &Tc); /* T_1 = I */
    else {
      rc = csr_mul(&h->T[l], &h->P[l], &TP);
      if (!rc) rc = csr_mul(&h->PH[l], &TP, &Tc);
      csr_free(&TP);
    }
    if (!rc) rc = csr_symmetrise(&Tc, 0);
    if (rc) return rc;
    csr_free(&h->T[l + 1]);
    h->T[l + 1] = Tc;
  }
  if (l + 1 == h->L - 1) rc = hier_coarsest_lu(h);
  return rc;
}

int or_galerkin(const or_hier *hc, int l, cplx *Ac_stencil) {
  if (l < 0 || l + 1 >= hc->L) return OR_EINVAL;
  or_csr AP, Ac;
  int rc = csr_mul(&hc->A[l], &hc->P[l], &AP);
  if (rc) return rc;
  rc = csr_mul(&hc->PH[l], &AP, &Ac);
  csr_free(&AP);
  if (!rc) rc = csr_to_stencil(hc->N[l + 1], &Ac, Ac_stencil);
  csr_free(&Ac);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Bootstrap setup (Secs. 3.4, 3.5, 4.1; Fig. 3.2 W-cycle scheme).          */
/* All work is on Z_l = Gamma5 D_l (Thm. 3.1): Kaczmarz on D_l v = b is the  */
/* same as on Z_l, the Ritz value is Eq. (3.17).                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  or_hier *h;
  const or_setup_params *p;
  int kr, ke;
  cplx *Vr[OR_MAXLEV], *Ve[OR_MAXLEV];
  double *lr[OR_MAXLEV], *le[OR_MAXLEV];
  int have_e[OR_MAXLEV];
  double *ritz_fine;
} setup_state;

static int lev_n(const or_hier *h, int l) { return h->A[l].nrow; }

/* <T_l v, v> (T_0 = I) */
static double t_norm2(const or_hier *h, int l, const cplx *v) {
  int n = lev_n(h, l);
  if (l == 0) return creal(vdot(n, v, v));
  cplx *t = malloc(sizeof(cplx) * n);
  csr_matvec(&h->T[l], v, t);
  double r = creal(vdot(n, v, t));
  free(t);
  return r;
}

/* Eq. (3.17): lambda = <Z v, v> / <T v, v>, Z = Gamma5 A (gamma5 = diag(1,-1)
 * per site) */
static double ritz(const or_hier *h, int l, const cplx *v) {
  int n = lev_n(h, l);
  cplx *t = malloc(sizeof(cplx) * n);
  csr_matvec(&h->A[l], v, t);
  cplx s = 0;
  for (int i = 0; i < n; ++i) s += conj(v[i]) * ((i & 1) ? -t[i] : t[i]);
  free(t);
  return creal(s) / t_norm2(h, l, v);
}

/* Eq. (3.6): Kaczmarz on D_l v = 0 */
static int relax_homog(const or_hier *h, int l, cplx *v, int sweeps) {
  int n = lev_n(h, l);
  cplx *r = malloc(sizeof(cplx) * n);
  if (!r) return OR_ENOMEM;
  csr_matvec(&h->A[l], v, r);
  for (int i = 0; i < n; ++i) r[i] = -r[i];
  int rc = or_kaczmarz(h, l, v, r, (h->N[l] % 8) ? OR_ORDER_LEX : OR_ORDER_COLOUR, sweeps, 1.0, NULL);
  free(r);
  return rc;
}

/* Eqs. (3.10)-(3.12) via Thm. 3.1 (ii): Kaczmarz on D_l v = lam Gamma5 T_l v.
 * Reading: the right-hand side is frozen within a sweep and lam is updated
 * after every sweep; v is T-normalised after the sweeps. */
static int relax_eig(const or_hier *h, int l, cplx *v, double *lam, int sweeps) {
  int n = lev_n(h, l);
  cplx *r = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
  if (!r || !t) { free(r); free(t); return OR_ENOMEM; }
  int rc = OR_OK;
  for (int sw = 0; sw < sweeps && !rc; ++sw) {
    if (l == 0) memcpy(t, v, sizeof(cplx) * n);
    else csr_matvec(&h->T[l], v, t);
    csr_matvec(&h->A[l], v, r);
    for (int i = 0; i < n; ++i) r[i] = (*lam) * ((i & 1) ? -t[i] : t[i]) - r[i];
    rc = or_kaczmarz(h, l, v, r, (h->N[l] % 8) ? OR_ORDER_LEX : OR_ORDER_COLOUR, 1, 1.0, NULL);
    *lam = ritz(h, l, v);
  }
  double nn = sqrt(t_norm2(h, l, v));
  if (nn > 0) for (int i = 0; i < n; ++i) v[i] /= nn;
  free(r); free(t);
  return rc;
}

/* Reading: a test vector is carried to the next coarser grid by its values
 * at the C points (the C rows of P are the identity, so v ~ P v_c). */
static void inject(const or_hier *h, int l, const cplx *v, cplx *vc) {
  int Nc = h->N[l + 1], nc = n_sites(Nc);
  for (int hc = 0; hc < nc; ++hc) {
    int hf = c_point(Nc, h->B[l], hc);
    vc[2 * hc] = v[2 * hf];
    vc[2 * hc + 1] = v[2 * hf + 1];
  }
}

/* Sec. 3.3 / reading of the weights promised there: every test vector is
 * T-normalised and weighted by 1 / max(|lambda|, 1e-12) with its Ritz value
 * (Eq. 3.17), so near-kernel vectors dominate the fit. */
static int fit_level(setup_state *S, int l) {
  or_hier *h = S->h;
  int n = lev_n(h, l);
  int k = S->kr + (S->have_e[l] ? S->ke : 0);
  cplx *V = malloc(sizeof(cplx) * (size_t)n * k);
  double *w = malloc(sizeof(double) * k);
  cplx *Pw = malloc(sizeof(cplx) * (size_t)n_sites(h->N[l]) * 8);
  if (!V || !w || !Pw) { free(V); free(w); free(Pw); return OR_ENOMEM; }
  for (int q = 0; q < k; ++q) {
    const cplx *src = q < S->kr ? S->Vr[l] + (size_t)q * n : S->Ve[l] + (size_t)(q - S->kr) * n;
    double nn = sqrt(t_norm2(h, l, src));
    for (int i = 0; i < n; ++i) V[(size_t)q * n + i] = nn > 0 ? src[i] / nn : 0;
    double lam = ritz(h, l, V + (size_t)q * n);
    w[q] = 1.0 / fmax(fabs(lam), 1e-12);
  }
  int rc = or_ls_fit(h->N[l], h->B[l], k, V, w, Pw);
  if (!rc) {
    csr_free(&h->P[l]);
    csr_free(&h->PH[l]);
    rc = build_P(h->N[l], h->B[l], Pw, &h->P[l]);
  }
  if (!rc) rc = csr_transpose(&h->P[l], 1, &h->PH[l]);
  if (!rc) rc = galerkin_level(h, l);
  free(V); free(w); free(Pw);
  return rc;
}

static int coarsest_eig(setup_state *S) {
  or_hier *h = S->h;
  int l = h->L - 1, n = lev_n(h, l);
  cplx *Z = malloc(sizeof(cplx) * (size_t)n * n), *T = malloc(sizeof(cplx) * (size_t)n * n);
  cplx *V = malloc(sizeof(cplx) * (size_t)n * n);
  double *lam = malloc(sizeof(double) * n);
  int *ord = malloc(sizeof(int) * n);
  if (!Z || !T || !V || !lam || !ord) { free(Z); free(T); free(V); free(lam); free(ord); return OR_ENOMEM; }
  or_csr_dense(&h->A[l], Z);
  for (int i = 0; i < n; ++i)
    if (i & 1) for (int j = 0; j < n; ++j) Z[(size_t)i * n + j] = -Z[(size_t)i * n + j];
  or_csr_dense(&h->T[l], T);
  int rc = or_gen_eig(n, Z, T, lam, V);
  if (!rc) {
    /* k_e eigenpairs with the smallest |lambda| (Sec. 3.4) */
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 1; i < n; ++i) {
      int t = ord[i], j = i - 1;
      while (j >= 0 && fabs(lam[ord[j]]) > fabs(lam[t])) { ord[j + 1] = ord[j]; j--; }
      ord[j + 1] = t;
    }
    for (int e = 0; e < S->ke; ++e) {
      memcpy(S->Ve[l] + (size_t)e * n, V + (size_t)ord[e] * n, sizeof(cplx) * n);
      S->le[l][e] = lam[ord[e]];
    }
    S->have_e[l] = 1;
  }
  free(Z); free(T); free(V); free(lam); free(ord);
  return rc;
}

static int interp_e(setup_state *S, int l) { /* Ve[l] = P Ve[l+1] */
  or_hier *h = S->h;
  int n = lev_n(h, l), nc = lev_n(h, l + 1);
  for (int e = 0; e < S->ke; ++e) {
    csr_matvec(&h->P[l], S->Ve[l + 1] + (size_t)e * nc, S->Ve[l] + (size_t)e * n);
    S->le[l][e] = S->le[l + 1][e];
  }
  S->have_e[l] = 1;
  return OR_OK;
}

static void inject_all(setup_state *S, int l) {
  or_hier *h = S->h;
  int n = lev_n(h, l), nc = n_sites(h->N[l + 1]) * 2;
  for (int q = 0; q < S->kr; ++q) inject(h, l, S->Vr[l] + (size_t)q * n, S->Vr[l + 1] + (size_t)q * nc);
  if (S->have_e[l]) {
    for (int e = 0; e < S->ke; ++e) {
      inject(h, l, S->Ve[l] + (size_t)e * n, S->Ve[l + 1] + (size_t)e * nc);
      S->le[l + 1][e] = S->le[l][e];
    }
    S->have_e[l + 1] = 1;
  }
}

static int relax_both(setup_state *S, int l, int mu, int with_e) {
  int n = lev_n(S->h, l), rc = OR_OK;
  for (int q = 0; q < S->kr && !rc; ++q) rc = relax_homog(S->h, l, S->Vr[l] + (size_t)q * n, mu);
  if (with_e && S->have_e[l])
    for (int e = 0; e < S->ke && !rc; ++e) rc = relax_eig(S->h, l, S->Ve[l] + (size_t)e * n, &S->le[l][e], mu);
  return rc;
}

/* One visit of level l >= 1 inside the W-cycle setup (Fig. 3.2): pre node,
 * first coarse visit, middle node (interpolate V^e, relax both sets,
 * recompute P), second coarse visit, post node (interpolate V^e, relax V^e).
 * At the coarsest level: generalised eigensolve (Thm. 3.1 (i)). */
static int setup_visit(setup_state *S, int l, int first, int mu) {
  or_hier *h = S->h;
  if (l == h->L - 1) return coarsest_eig(S);
  int rc = relax_both(S, l, mu, !first);
  if (!rc) rc = fit_level(S, l);
  if (!rc) inject_all(S, l);
  if (!rc) rc = setup_visit(S, l + 1, first, mu);
  if (!rc) rc = interp_e(S, l);
  if (!rc) rc = relax_both(S, l, mu, 1);
  if (!rc) rc = fit_level(S, l);
  if (!rc) inject_all(S, l);
  if (!rc) rc = setup_visit(S, l + 1, 0, mu);
  if (!rc) rc = interp_e(S, l);
  for (int e = 0; e < S->ke && !rc; ++e)
    rc = relax_eig(h, l, S->Ve[l] + (size_t)e * lev_n(h, l), &S->le[l][e], mu);
  return rc;
}

/* Sec. 4.2 super-V setup cycle: every grid is visited once and the coarsest
 * eigensolve runs once per setup cycle; grid l >= 1 relaxes mu 2^l times
 * before (both vector sets, then fit and injection) and after (the
 * eigenvector set, Eq. 3.16) its coarse visit.  Reading: this gives each
 * grid the relaxation count of the W-visits above (2^(l-1) visits with mu
 * sweeps at each of the pre, middle and post nodes) in V(mu 2^l, mu 2^l)
 * form; P of grid l is the one fitted before its coarse visit. */
static int setup_visit_superv(setup_state *S, int l, int first, int mu) {
  or_hier *h = S->h;
  if (l == h->L - 1) return coarsest_eig(S);
  int mul = mu << l;
  int rc = relax_both(S, l, mul, !first);
  if (!rc) rc = fit_level(S, l);
  if (!rc) inject_all(S, l);
  if (!rc) rc = setup_visit_superv(S, l + 1, first, mu);
  if (!rc) rc = interp_e(S, l);
  for (int e = 0; e < S->ke && !rc; ++e)
    rc = relax_eig(h, l, S->Ve[l] + (size_t)e * lev_n(h, l), &S->le[l][e], mul);
  return rc;
}

/* Sec. 4.1 adaptive step: the test vector on the finest grid with the
 * smallest |lambda| (Eq. 3.17) is improved by two solver cycles applied to
 * D_1 v = 0 (x <- x + M(0 - A x)). */
static int adaptive_step(setup_state *S) {
  or_hier *h = S->h;
  int n = lev_n(h, 0), best = -1;
  double bl = INFINITY;
  int k = S->kr + (S->have_e[0] ? S->ke : 0);
  for (int q = 0; q < k; ++q) {
    cplx *v = q < S->kr ? S->Vr[0] + (size_t)q * n : S->Ve[0] + (size_t)(q - S->kr) * n;
    double lam = fabs(ritz(h, 0, v));
    if (lam < bl) { bl = lam; best = q; }
  }
  if (best < 0) return OR_OK;
  cplx *v = best < S->kr ? S->Vr[0] + (size_t)best * n : S->Ve[0] + (size_t)(best - S->kr) * n;
  cplx *r = malloc(sizeof(cplx) * n), *e = malloc(sizeof(cplx) * n);
  if (!r || !e) { free(r); free(e); return OR_ENOMEM; }
  int rc = OR_OK;
  for (int it = 0; it < 2 && !rc; ++it) {
    csr_matvec(&h->A[0], v, r);
    for (int i = 0; i < n; ++i) r[i] = -r[i];
    rc = or_cycle(h, 0, r, e, S->p->nu_pre, S->p->nu_post, S->p->gamma, OR_ORDER_COLOUR);
    for (int i = 0; i < n && !rc; ++i) v[i] += e[i];
  }
  double nn = sqrt(t_norm2(h, 0, v));
  if (nn > 0) for (int i = 0; i < n; ++i) v[i] /= nn;
  if (best >= S->kr) S->le[0][best - S->kr] = ritz(h, 0, v);
  free(r); free(e);
  return rc;
}

/* Secs. 3.4 and 4.1: first setup cycle (relaxation mu1; initial hierarchy
 * from k_r random vectors only), adaptive step, second setup cycle (mu2). */
or_hier *or_setup(int N, const cplx *U, double m, const or_setup_params *p,
                  double *ritz_out) {
  int L = p->levels;
  int Nl[OR_MAXLEV], Bl[OR_MAXLEV];
  if (L < 2 || L > OR_MAXLEV || p->k_r < 1 || p->k_e < 0) return NULL;
  Nl[0] = N;
  for (int l = 0; l + 1 < L; ++l) { Bl[l] = p->block[l]; Nl[l + 1] = Nl[l] / (Bl[l] > 0 ? Bl[l] : 1); }
  Bl[L - 1] = 0;
  if (check_levels(N, L, Nl, Bl)) return NULL;
  or_hier *h = calloc(1, sizeof(or_hier));
  if (!h) return NULL;
  h->L = L;
  h->Nfine = N;
  h->m = m;
  h->nT = 1;
  for (int l = 0; l < L; ++l) { h->N[l] = Nl[l]; h->B[l] = Bl[l]; }
  setup_state S;
  memset(&S, 0, sizeof(S));
  S.h = h;
  S.p = p;
  S.kr = p->k_r;
  S.ke = p->k_e;
  int rc = dhat_matrix(N, U, m, &h->A[0]);
  if (!rc) rc = csr_transpose(&h->A[0], 0, &h->AT[0]);
  for (int l = 0; l < L && !rc; ++l) {
    size_t n = (size_t)n_sites(Nl[l]) * 2;
    S.Vr[l] = calloc(n * S.kr, sizeof(cplx));
    S.Ve[l] = calloc(n * (S.ke ? S.ke : 1), sizeof(cplx));
    S.lr[l] = calloc(S.kr, sizeof(double));
    S.le[l] = calloc(S.ke ? S.ke : 1, sizeof(double));
    if (!S.Vr[l] || !S.Ve[l] || !S.lr[l] || !S.le[l]) rc = OR_ENOMEM;
  }
  if (!rc) {
    size_t n0 = (size_t)n_sites(N) * 2;
    for (int q = 0; q < S.kr; ++q)
      for (size_t i = 0; i < n0; ++i) S.Vr[0][q * n0 + i] = or_rng_cgauss(p->seed, (uint64_t)q, i);
  }
  /* cycle 1: black pre node on the finest grid, W-visit of level 1, white node */
  if (!rc) rc = relax_both(&S, 0, p->mu1, 0);
  if (!rc) rc = fit_level(&S, 0);
  if (!rc) inject_all(&S, 0);
  if (!rc) rc = p->setup_cycle == 1 ? setup_visit_superv(&S, 1, 1, p->mu1) : setup_visit(&S, 1, 1, p->mu1);
  if (!rc) rc = interp_e(&S, 0);
  if (!rc) rc = adaptive_step(&S);
  /* cycle 2: green pre node on the finest grid, W-visit of level 1 */
  if (!rc) rc = relax_both(&S, 0, p->mu2, 1);
  if (!rc) rc = fit_level(&S, 0);
  if (!rc) inject_all(&S, 0);
  if (!rc) rc = p->setup_cycle == 1 ? setup_visit_superv(&S, 1, 0, p->mu2) : setup_visit(&S, 1, 0, p->mu2);
  if (!rc) rc = interp_e(&S, 0);
  if (!rc && ritz_out)
    for (int e = 0; e < S.ke; ++e) ritz_out[e] = S.le[0][e];
  for (int l = 0; l < L; ++l) { free(S.Vr[l]); free(S.Ve[l]); free(S.lr[l]); free(S.le[l]); }
  if (rc) { or_hier_free(h); return NULL; }
  return h;
}

/* ------------------------------------------------------------------------ */
/* Aggregation coarse space.  Sec. 4 closes by naming the alternative to its */
/* W-cycles that it did not explore: more interpolation variables per coarse */
/* point.  Reading used here (the aggregation-based solvers the paper cites   */
/* as related work): the aggregates are the B x B cells of the full          */
/* coarsening (Sec. 3.2 reading: the cell with corner (a0, b0) = (B floor(a/B),*/
/* B floor(b/B)) holds the fine sites (a0 + ia, b0 + ib), 0 <= ia, ib < B,    */
/* member index ia B + ib); for every aggregate and spin s the k test vectors */
/* restricted to (aggregate, spin s) are orthonormalised by modified         */
/* Gram-Schmidt in their given order, and those k columns are the columns of  */
/* P for that (aggregate, spin).  Coarse variable 2k hc + k s + kappa of the  */
/* coarse site hc (the cell's corner on the N/B lattice).  P is block        */
/* diagonal in spin, so Gamma5 P = P Gamma5c with Gamma5c = +1 on the first k */
/* variables of a coarse site and -1 on the last k, and the Galerkin operator */
/* P^H A P (Sec. 3.5) is Gamma5c-Hermitian.  A fine site couples (3 x 3 box  */
/* in (a, b)) only to sites of its own or an adjacent cell, so P^H A P is a   */
/* 9-point stencil of dense 2k x 2k blocks on the coarse lattice.            */
/* ------------------------------------------------------------------------ */
static void agg_member(int N, int B, int h, int *hc, int *m) {
  int x, y;
  site_xy(N, h, &x, &y);
  int a = (x + y) / 2, b = (x - y) / 2;
  int a0 = B * floordiv(a, B), b0 = B * floordiv(b, B);
  int xc = wrap(a0 + b0, N), yc = wrap(a0 - b0, N);
  *hc = site_of(N / B, xc / B, yc / B);
  *m = (a - a0) * B + (b - b0);
}

/* Q[hc][s][m][kappa] from the k test vectors V[kappa][2 nf] of a level-N
 * lattice (unknown 2 h + s).  OR_ESTRUCT if some (aggregate, spin) block of
 * the test vectors has rank < k (modified Gram-Schmidt leaves a column of
 * norm <= 1e-12 times the column it started from). */
int or_agg_interp(int N, int B, int k, const cplx *V, cplx *Q) {
  if (B < 2 || N % B || (N / 2) % B || k < 1 || k > B * B) return OR_EINVAL;
  int nf = n_sites(N), nc = n_sites(N / B), M = B * B;
  for (int h = 0; h < nf; ++h) {
    int hc, m;
    agg_member(N, B, h, &hc, &m);
    for (int s = 0; s < 2; ++s)
      for (int kap = 0; kap < k; ++kap)
        Q[(((size_t)hc * 2 + s) * M + m) * k + kap] = V[(size_t)kap * 2 * nf + 2 * h + s];
  }
  for (int hc = 0; hc < nc; ++hc)
    for (int s = 0; s < 2; ++s) {
      cplx *q = Q + ((size_t)hc * 2 + s) * M * k; /* q[m * k + kappa] */
      for (int kap = 0; kap < k; ++kap) {
        double n0 = 0;
        for (int m = 0; m < M; ++m) n0 += creal(q[m * k + kap] * conj(q[m * k + kap]));
        for (int lam = 0; lam < kap; ++lam) {
          cplx d = 0; /* q_lambda^H q_kappa */
          for (int m = 0; m < M; ++m) d += conj(q[m * k + lam]) * q[m * k + kap];
          for (int m = 0; m < M; ++m) q[m * k + kap] -= d * q[m * k + lam];
        }
        double nn = 0;
        for (int m = 0; m < M; ++m) nn += creal(q[m * k + kap] * conj(q[m * k + kap]));
        if (!(sqrt(nn) > 1e-12 * sqrt(n0))) return OR_ESTRUCT;
        for (int m = 0; m < M; ++m) q[m * k + kap] /= sqrt(nn);
      }
    }
  return OR_OK;
}

static int agg_P_csr(int N, int B, int k, const cplx *Q, or_csr *P) {
  int nf = n_sites(N), nc = n_sites(N / B), M = B * B;
  triplets t = {0};
  int rc = OR_OK;
  for (int h = 0; h < nf && !rc; ++h) {
    int hc, m;
    agg_member(N, B, h, &hc, &m);
    for (int s = 0; s < 2 && !rc; ++s)
      for (int kap = 0; kap < k && !rc; ++kap)
        rc = trip_push(&t, 2 * h + s, 2 * k * hc + k * s + kap, Q[(((size_t)hc * 2 + s) * M + m) * k + kap]);
  }
  if (!rc) rc = csr_from_triplets(2 * nf, 2 * k * nc, &t, P);
  trip_free(&t);
  return rc;
}

/* Galerkin operator of level l of h with the aggregation P of Q:
 * Ac[hc][d][r][c] (2k x 2k blocks, offset d as for the stencils above) =
 * (P^H A_l P) restricted to the coarse sites hc and neighbour(hc, d). */
int or_agg_galerkin(const or_hier *h, int l, int B, int k, const cplx *Q, cplx *Ac) {
  if (l < 0 || l >= h->L) return OR_EINVAL;
  int N = h->N[l], Nc = N / B, nc = n_sites(Nc), K2 = 2 * k;
  if (B < 2 || N % B || (N / 2) % B || Nc < 8) return OR_EINVAL;
  or_csr P = {0}, PH = {0}, AP = {0}, C = {0};
  int rc = agg_P_csr(N, B, k, Q, &P);
  if (!rc) rc = csr_transpose(&P, 1, &PH);
  if (!rc) rc = csr_mul(&h->A[l], &P, &AP);
  if (!rc) rc = csr_mul(&PH, &AP, &C);
  if (!rc) {
    memset(Ac, 0, sizeof(cplx) * (size_t)nc * 9 * K2 * K2);
    for (int row = 0; row < C.nrow && !rc; ++row) {
      int hr = row / K2, r = row % K2;
      for (int p = C.rowptr[row]; p < C.rowptr[row + 1]; ++p) {
        int hcol = C.col[p] / K2, c = C.col[p] % K2, found = 0;
        for (int d = 0; d < 9; ++d)
          if (or_stencil_neighbour(Nc, hr, d) == hcol) {
            Ac[(((size_t)hr * 9 + d) * K2 + r) * K2 + c] += C.val[p];
            found = 1;
            break;
          }
        if (!found && C.val[p] != 0) rc = OR_ESTRUCT;
      }
    }
  }
  csr_free(&P); csr_free(&PH); csr_free(&AP); csr_free(&C);
  return rc;
}

/* y = Ac x on the coarse lattice Nc (x, y [nc][2k]): y_h = sum_d Ac[h][d] x_{neighbour(h, d)}. */
int or_agg_apply(int Nc, int k, const cplx *Ac, const cplx *x, cplx *y) {
  int nc = n_sites(Nc), K2 = 2 * k;
  for (int h = 0; h < nc; ++h)
    for (int r = 0; r < K2; ++r) {
      cplx s = 0;
      for (int d = 0; d < 9; ++d) {
        int j = or_stencil_neighbour(Nc, h, d);
        for (int c = 0; c < K2; ++c) s += Ac[(((size_t)h * 9 + d) * K2 + r) * K2 + c] * x[(size_t)j * K2 + c];
      }
      y[(size_t)h * K2 + r] = s;
    }
  return OR_OK;
}

/* fc = P^H r (r a level-N vector [2 nf], fc [nc][2k]) and x += P e. */
int or_agg_restrict(int N, int B, int k, const cplx *Q, const cplx *r, cplx *fc) {
  int nf = n_sites(N), nc = n_sites(N / B), M = B * B;
  memset(fc, 0, sizeof(cplx) * (size_t)nc * 2 * k);
  for (int h = 0; h < nf; ++h) {
    int hc, m;
    agg_member(N, B, h, &hc, &m);
    for (int s = 0; s < 2; ++s)
      for (int kap = 0; kap < k; ++kap)
        fc[(size_t)hc * 2 * k + k * s + kap] += conj(Q[(((size_t)hc * 2 + s) * M + m) * k + kap]) * r[2 * h + s];
  }
  return OR_OK;
}

int or_agg_prolong(int N, int B, int k, const cplx *Q, const cplx *e, cplx *x) {
  int nf = n_sites(N), M = B * B;
  for (int h = 0; h < nf; ++h) {
    int hc, m;
    agg_member(N, B, h, &hc, &m);
    for (int s = 0; s < 2; ++s) {
      cplx t = 0;
      for (int kap = 0; kap < k; ++kap)
        t += Q[(((size_t)hc * 2 + s) * M + m) * k + kap] * e[(size_t)hc * 2 * k + k * s + kap];
      x[2 * h + s] += t;
    }
  }
  return OR_OK;
}

/* Host threads the loops above run on: 1 in the plain build. */
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
