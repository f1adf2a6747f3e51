// wl_setup.cu -- bootstrap AMG setup on the GPU (Secs. 3.3-3.5, 4.1).
//
// The k test vectors of a level are held as one batch [n][2][k] (vector
// index innermost, like right-hand sides), so homogeneous relaxation
// (Eq. 3.6) and the eigen-relaxation of Thm. 3.1 (ii) reuse the solve-phase
// Kaczmarz kernel.  Setup-only kernels: least-squares interpolation
// (Eq. 3.4), Galerkin triple products P^H A P and P^H T P (Sec. 3.5),
// injection to C points, Ritz values (Eq. 3.17), and the coarsest
// generalised Hermitian eigenproblem Z_L v = lambda T_L v (Thm. 3.1 (i),
// cuSOLVER zhegvd).  Schedule: W-cycle setup of Fig. 3.2 with setup_mu[0]
// sweeps, the adaptive step of Sec. 4.1, a second W-cycle with setup_mu[1].
#include <cusolverDn.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "wl_common.cuh"

namespace wl {
int resolve_levels(int N, amg_params *p, int *Nl);
int hier_alloc(wl_amg *a, const int *Nl);
int hier_finish(wl_amg *a);
void amg_free(wl_amg *a);
int cycle_direct(wl_amg *a, int nrhs, int prec, cudaStream_t s);
}

// ------------------------------------------------------------ random start
// SplitMix64 output function on a counter (Steele, Lea & Flood 2014):
// u64(seed, stream, i) = sm(sm(sm(seed) + stream) + i); Box-Muller on
// uniforms ((u >> 11) + 1) 2^-53 at counters 2i and 2i+1.
__host__ __device__ __forceinline__ unsigned long long sm64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void k_random_vectors(long n2, int k, unsigned long long seed, zd *V) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n2 * k) return;
  long i = tid / k;
  int q = (int)(tid - i * k);
  unsigned long long key = sm64(sm64(seed) + (unsigned long long)q);
  unsigned long long u1 = sm64(key + 2ULL * (unsigned long long)i);
  unsigned long long u2 = sm64(key + 2ULL * (unsigned long long)i + 1ULL);
  double f1 = ((double)(u1 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
  double f2 = ((double)(u2 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
  double r = sqrt(-2.0 * log(f1));
  double s, c;
  sincospi(2.0 * f2, &s, &c);
  V[tid] = mk(r * c, r * s);
}

// ------------------------------------------------------------ small kernels
__global__ void k_g5_inplace(zd *v, long n, int k) {  // negate spin-1 entries
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n * k) return;
  long h = tid / k;
  int q = (int)(tid - h * k);
  zd &e = v[(h * 2 + 1) * k + q];
  e = mk(-e.re, -e.im);
}

// out[i][s][q] = coef[q] * gamma5_s * in[i][s][q]  (g5 = 0: without the sign)
__global__ void k_scale_vec(const zd *in, zd *out, const double *coef, long n, int k, int g5) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n * 2 * k) return;
  int q = (int)(tid % k);
  int s = (int)((tid / k) & 1);
  double f = coef[q] * ((g5 && s) ? -1.0 : 1.0);
  out[tid] = f * in[tid];
}

// gather (Vr, Ve) into one normalised batch W with scale factors
__global__ void k_gather_tv(const zd *Vr, int kr, const zd *Ve, int ke, const double *scale, zd *W, long n2) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int k = kr + ke;
  if (tid >= n2 * k) return;
  long i = tid / k;
  int q = (int)(tid - i * k);
  zd v = q < kr ? Vr[i * kr + q] : Ve[i * ke + (q - kr)];
  W[tid] = scale[q] * v;
}

// value of a test vector at the C points: vc[hc][s][q] = v[cpoint(hc)][s][q]
__global__ void k_inject(Geo gf, Geo gc, int lgB, const zd *v, zd *vc, int k) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int nc = gc.nsites();
  if (tid >= (long)nc * k) return;
  int hc = (int)(tid / k), q = (int)(tid - (long)hc * k);
  int xc, yc;
  gc.xy(hc, xc, yc);
  int hf = gf.idx(xc << lgB, yc << lgB);
  vc[((long)hc * 2) * k + q] = v[((long)hf * 2) * k + q];
  vc[((long)hc * 2 + 1) * k + q] = v[((long)hf * 2 + 1) * k + q];
}

// identity stencil (T_0 = I)
__global__ void k_identity_stencil(int n, zd *T) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long)n * 36) return;
  int e = (int)(tid % 36);
  int d = e / 4, st = e % 4;
  T[tid] = mk((d == 4 && (st == 0 || st == 3)) ? 1.0 : 0.0, 0.0);
}

// cell corners of fine site (x, y): coarse index per corner k (-1 if absent)
__device__ __forceinline__ void corners(const Geo &gf, const Geo &gc, int lgB, int px, int py, int ck[4]) {
  int B = 1 << lgB;
  int a = (px + py) >> 1, b = (px - py) >> 1;
  int a0 = a & ~(B - 1), b0 = b & ~(B - 1);
  int ra = a - a0, rb = b - b0;
  for (int k = 0; k < 4; ++k) {
    int ka = k & 1, kb = k >> 1;
    if ((ka && !ra) || (kb && !rb)) {
      ck[k] = -1;
      continue;
    }
    int ac = a0 + ka * B, bc = b0 + kb * B;
    int xf = (ac + bc) & (gf.N - 1), yf = (ac - bc) & (gf.N - 1);
    ck[k] = gc.idx(xf >> lgB, yf >> lgB);
  }
}

// Hermitian Jacobi on n <= 4 (row major), eigenvectors in columns of Q
__device__ void jacobi4(int n, zd *A, zd *Q, double *lam) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Q[i * 4 + j] = mk(i == j ? 1.0 : 0.0, 0.0);
  double fro = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) fro += cnorm2(A[i * 4 + j]);
  fro = sqrt(fro);
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += cnorm2(A[p * 4 + q]);
    if (sqrt(off) <= 1e-16 * fro || fro == 0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        zd apq = A[p * 4 + q];
        double ab = sqrt(cnorm2(apq));
        if (ab == 0.0) continue;
        zd e = mk(apq.re / ab, apq.im / ab);
        double tau = (A[q * 4 + q].re - A[p * 4 + p].re) / (2.0 * ab);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        zd se = s * e, sec = s * cconj(e);
        for (int k = 0; k < n; ++k) {
          zd akp = A[k * 4 + p], akq = A[k * 4 + q];
          A[k * 4 + p] = c * akp - sec * akq;
          A[k * 4 + q] = se * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          zd apk = A[p * 4 + k], aqk = A[q * 4 + k];
          A[p * 4 + k] = c * apk - se * aqk;
          A[q * 4 + k] = sec * apk + c * aqk;
        }
        A[p * 4 + q] = mk(0.0, 0.0);
        A[q * 4 + p] = mk(0.0, 0.0);
        A[p * 4 + p].im = 0;
        A[q * 4 + q].im = 0;
        for (int k = 0; k < n; ++k) {
          zd qkp = Q[k * 4 + p], qkq = Q[k * 4 + q];
          Q[k * 4 + p] = c * qkp - sec * qkq;
          Q[k * 4 + q] = se * qkp + c * qkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i * 4 + i].re;
}

// Eq. 3.4 for every fine variable (h, s): minimise sum_q w_q |v_i - sum_j
// p_j v_j|^2 over the same-spin cell corners j; normal equations M p = g
// with M_ab = sum_q w_q conj(v_a) v_b, g_a = sum_q w_q conj(v_a) v_i,
// eigen-pseudoinverse dropping eigenvalues <= 1e-12 trace(M).  C points get
// the identity row.  W is the test-vector batch [n][2][k].
__global__ void k_ls_fit(Geo gf, Geo gc, int lgB, const zd *__restrict__ W, const double *__restrict__ w,
                         int k, zd *__restrict__ P) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int nf = gf.nsites();
  if (tid >= 2 * nf) return;
  int h = tid >> 1, s = tid & 1;
  int px, py;
  gf.xy(h, px, py);
  int ck[4];
  corners(gf, gc, lgB, px, py, ck);
  zd *out = P + (long)h * 8 + s * 4;
  int idx[4], cf[4], nc = 0;
  for (int q = 0; q < 4; ++q)
    if (ck[q] >= 0) {
      idx[nc] = q;
      int xc, yc;
      gc.xy(ck[q], xc, yc);
      cf[nc] = gf.idx(xc << lgB, yc << lgB);
      nc++;
    }
  for (int q = 0; q < 4; ++q) out[q] = mk(0.0, 0.0);
  if (nc == 1) {
    out[0] = mk(1.0, 0.0);
    return;
  }
  zd M[16], g[4], Q[16];
  double mu[4];
  for (int a = 0; a < 4; ++a) {
    g[a] = mk(0.0, 0.0);
    for (int b = 0; b < 4; ++b) M[a * 4 + b] = mk(0.0, 0.0);
  }
  for (int q = 0; q < k; ++q) {
    double wq = w[q];
    zd vi = W[((long)h * 2 + s) * k + q];
    zd va[4];
    for (int a = 0; a < nc; ++a) va[a] = W[((long)cf[a] * 2 + s) * k + q];
    for (int a = 0; a < nc; ++a) {
      zd t = cmulc(va[a], vi);
      g[a] = g[a] + wq * t;
      for (int b = 0; b < nc; ++b) M[a * 4 + b] = M[a * 4 + b] + wq * cmulc(va[a], va[b]);
    }
  }
  double tr = 0;
  for (int a = 0; a < nc; ++a) tr += M[a * 4 + a].re;
  jacobi4(nc, M, Q, mu);
  zd p[4] = {mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0)};
  for (int e = 0; e < nc; ++e) {
    if (mu[e] <= 1e-12 * tr) continue;
    zd qg = mk(0.0, 0.0);
    for (int a = 0; a < nc; ++a) qg = qg + cmulc(Q[a * 4 + e], g[a]);
    for (int a = 0; a < nc; ++a) p[a] = p[a] + (1.0 / mu[e]) * (Q[a * 4 + e] * qg);
  }
  for (int a = 0; a < nc; ++a) out[idx[a]] = p[a];
}

// Galerkin block (hc, d): sum over fine i in the box of hc and fine
// neighbours j of i whose cell has nb(hc, d) as a corner:
//   Ac[hc][d][s][t] = sum conj(P[i][s][k_i]) A[i][df][s][t] P[j][t][k_j]
__global__ void k_galerkin(Geo gf, Geo gc, int lgB, const zd *__restrict__ A, const zd *__restrict__ P,
                           zd *__restrict__ Ac) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int nc = gc.nsites();
  if (tid >= nc * 9) return;
  int hc = tid / 9, d = tid % 9;
  int xc, yc;
  gc.xy(hc, xc, yc);
  int cprime = gc.nb(xc, yc, d);
  int B = 1 << lgB;
  int X = xc << lgB, Y = yc << lgB;
  zd acc[2][2];
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) acc[s][t] = mk(0.0, 0.0);
  for (int da = -(B - 1); da <= B - 1; ++da)
    for (int db = -(B - 1); db <= B - 1; ++db) {
      int ix = X + da + db, iy = Y + da - db;
      int hi = gf.idx(ix, iy);
      int ki = (da < 0 ? 1 : 0) + (db < 0 ? 2 : 0);
      zd wi0 = P[(long)hi * 8 + ki], wi1 = P[(long)hi * 8 + 4 + ki];
      if (wi0.re == 0 && wi0.im == 0 && wi1.re == 0 && wi1.im == 0) continue;
      int ixw = ix & (gf.N - 1), iyw = iy & (gf.N - 1);
      for (int df = 0; df < 9; ++df) {
        int dfa = df / 3 - 1, dfb = df % 3 - 1;
        int jx = (ixw + dfa + dfb) & (gf.N - 1), jy = (iyw + dfa - dfb) & (gf.N - 1);
        int hj = gf.idx(jx, jy);
        int ck[4];
        corners(gf, gc, lgB, jx, jy, ck);
        for (int kj = 0; kj < 4; ++kj) {
          if (ck[kj] != cprime) continue;
          zd pj0 = P[(long)hj * 8 + kj], pj1 = P[(long)hj * 8 + 4 + kj];
          const zd *Ab = A + ((long)hi * 9 + df) * 4;
          zd ci0 = cconj(wi0), ci1 = cconj(wi1);
          acc[0][0] = acc[0][0] + ci0 * (Ab[0] * pj0);
          acc[0][1] = acc[0][1] + ci0 * (Ab[1] * pj1);
          acc[1][0] = acc[1][0] + ci1 * (Ab[2] * pj0);
          acc[1][1] = acc[1][1] + ci1 * (Ab[3] * pj1);
        }
      }
    }
  zd *o = Ac + ((long)hc * 9 + d) * 4;
  o[0] = acc[0][0];
  o[1] = acc[0][1];
  o[2] = acc[1][0];
  o[3] = acc[1][1];
}

// Hermitian part of a stencil (for T): X = (A_hd + A_j,8-d^H) / 2
__global__ void k_herm_stencil(Geo g, zd *A) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int n = g.nsites();
  if (tid >= n * 5) return;
  int h = tid / 5, q = tid % 5;
  int x, y;
  g.xy(h, x, y);
  if (q == 4) {
    zd *Bk = A + ((long)h * 9 + 4) * 4;
    zd b[4] = {Bk[0], Bk[1], Bk[2], Bk[3]};
    Bk[0] = mk(b[0].re, 0.0);
    Bk[3] = mk(b[3].re, 0.0);
    zd o = 0.5 * (b[1] + cconj(b[2]));
    Bk[1] = o;
    Bk[2] = cconj(o);
    return;
  }
  int d = 5 + q;
  int j = g.nb(x, y, d);
  zd *B1 = A + ((long)h * 9 + d) * 4;
  zd *B2 = A + ((long)j * 9 + (8 - d)) * 4;
  zd X[4];
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) X[s * 2 + t] = 0.5 * (B1[s * 2 + t] + cconj(B2[t * 2 + s]));
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) {
      B1[s * 2 + t] = X[s * 2 + t];
      B2[s * 2 + t] = cconj(X[t * 2 + s]);
    }
}

// dense column-major copy of a stencil operator (for cuSOLVER); g5 = 1
// multiplies row spin 1 by -1 (Z = Gamma5 A)
__global__ void k_stencil_dense_cm(Geo g, const zd *__restrict__ A, zd *M, int g5) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.nsites()) return;
  int n = 2 * g.nsites(), x, y;
  g.xy(h, x, y);
  for (int d = 0; d < 9; ++d) {
    int j = g.nb(x, y, d);
    for (int s = 0; s < 2; ++s)
      for (int t = 0; t < 2; ++t) {
        long o = (long)(2 * j + t) * n + 2 * h + s;  // column-major (row 2h+s, col 2j+t)
        zd v = A[((long)h * 9 + d) * 4 + s * 2 + t];
        if (g5 && s) v = mk(-v.re, -v.im);
        M[o] = M[o] + v;
      }
  }
}

// Ve[u][q] = Vcm[col_q * n + u]
__global__ void k_take_eigvecs(const zd *Vcm, int n, const int *cols, int ke, zd *Ve) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n * ke) return;
  int u = tid / ke, q = tid % ke;
  Ve[tid] = Vcm[(long)cols[q] * n + u];
}


__global__ void k_mdot_setup(const zd *u, const zd *v, long E, int R, zd *part) {
  extern __shared__ unsigned char sm_raw[];
  zd *sm = (zd *)sm_raw;
  int t = threadIdx.x, nt = blockDim.x;
  int G = nt / R, q = t / R;
  zd acc = mk(0.0, 0.0);
  for (long e = (long)blockIdx.x * nt + t; e < E; e += (long)gridDim.x * nt) cfmac(acc, u[e], v[e]);
  sm[t] = acc;
  __syncthreads();
  for (int s = G >> 1; s > 0; s >>= 1) {
    if (q < s) sm[t] = sm[t] + sm[t + s * R];
    __syncthreads();
  }
  if (q == 0) part[(long)blockIdx.x * R + t] = sm[t];
}

// ------------------------------------------------------------- host side
namespace {

struct SetupLevel {
  DBuf Vr, Ve, T, tmp1, tmp2, zero;
  std::vector<double> lam;  // Ritz values of Ve
  bool have_e = false;
};

struct Setup {
  wl_amg *a;
  int kr, ke;
  SetupLevel S[8];
  DBuf red, dots, coef, W, wts;
  cudaStream_t s;
  cusolverDnHandle_t cs = nullptr;
};

static int n2of(wl_amg *a, int l) { return a->lev[l].n * 2; }

// per-vector dots <u_q, v_q> over a batch [n2][k]; result host[k] (real parts)
static int batch_dots(Setup &S, const zd *u, const zd *v, long n2, int k, std::vector<double> &out) {
  cudaStream_t s = S.s;
  long E = n2 * k;
  int G = 1;
  while (k * G * 2 <= 256) G *= 2;
  int nt = k * G;
  int nblk = (int)std::max(1L, std::min((E + nt - 1) / nt, 1024L));
  std::vector<zd> h;
  // plain two-stage reduction on the device, final sum on the host in order
  WL_TRY(S.red.alloc(sizeof(zd) * (size_t)nblk * k));
  k_mdot_setup<<<nblk, nt, sizeof(zd) * nt, s>>>(u, v, E, k, S.red.as<zd>());
  WL_CUDA(cudaGetLastError());
  h.resize((size_t)nblk * k);
  WL_CUDA(cudaMemcpyAsync(h.data(), S.red.p, sizeof(zd) * h.size(), cudaMemcpyDeviceToHost, s));
  WL_CUDA(cudaStreamSynchronize(s));
  out.assign(k, 0.0);
  for (int b = 0; b < nblk; ++b)
    for (int q = 0; q < k; ++q) out[q] += h[(size_t)b * k + q].re;
  return WL_OK;
}


// T v (T_0 = I)
static int apply_T(Setup &S, int l, const zd *v, zd *out, int k) {
  wl_amg *a = S.a;
  long n2 = n2of(a, l);
  if (l == 0) {
    WL_CUDA(cudaMemcpyAsync(out, v, sizeof(zd) * n2 * k, cudaMemcpyDeviceToDevice, S.s));
    return WL_OK;
  }
  // reuse the FP64 stencil kernel through a temporary LevelOps view
  Level &L = a->lev[l];
  LevelOps save = L.op64;
  L.op64.A.p = S.S[l].T.p;
  int rc = wl::stencil_apply(a, l, WL_FP64, v, out, nullptr, k, S.s);
  L.op64 = save;
  return rc;
}

// lambda_q = <Gamma5 A v, v> / <T v, v> and <T v, v> for a batch
static int ritz(Setup &S, int l, const zd *v, int k, std::vector<double> &lam, std::vector<double> &tn) {
  wl_amg *a = S.a;
  long n2 = n2of(a, l);
  SetupLevel &SL = S.S[l];
  WL_TRY(wl::stencil_apply(a, l, WL_FP64, v, SL.tmp1.p, nullptr, k, S.s));
  k_g5_inplace<<<WL_GRID(n2 / 2 * k, 256), 256, 0, S.s>>>(SL.tmp1.as<zd>(), n2 / 2, k);
  std::vector<double> za;
  WL_TRY(batch_dots(S, v, SL.tmp1.as<zd>(), n2, k, za));
  WL_TRY(apply_T(S, l, v, SL.tmp2.as<zd>(), k));
  WL_TRY(batch_dots(S, v, SL.tmp2.as<zd>(), n2, k, tn));
  lam.resize(k);
  for (int q = 0; q < k; ++q) lam[q] = tn[q] > 0 ? za[q] / tn[q] : 0.0;
  return WL_OK;
}

// Eq. 3.6: Kaczmarz on A_l v = 0
static int relax_homog(Setup &S, int l, zd *V, int k, int sweeps) {
  if (sweeps <= 0 || k <= 0) return WL_OK;
  wl_amg *a = S.a;
  SetupLevel &SL = S.S[l];
  WL_TRY(wl::stencil_apply(a, l, WL_FP64, V, SL.tmp1.p, SL.zero.p, k, S.s));
  return wl::kaczmarz_sweeps(a, l, WL_FP64, V, SL.tmp1.p, k, sweeps, S.s);
}

// Thm. 3.1 (ii): Kaczmarz on A_l v = lambda Gamma5 T_l v, rhs frozen per
// sweep, lambda updated after each sweep (Eq. 3.17), T-normalised after
static int relax_eig(Setup &S, int l, int sweeps) {
  wl_amg *a = S.a;
  SetupLevel &SL = S.S[l];
  int k = S.ke;
  if (k <= 0 || !SL.have_e) return WL_OK;
  long n2 = n2of(a, l);
  zd *V = SL.Ve.as<zd>();
  std::vector<double> tn;
  WL_TRY(S.coef.alloc(sizeof(double) * 64));
  for (int sw = 0; sw < sweeps; ++sw) {
    WL_TRY(apply_T(S, l, V, SL.tmp2.as<zd>(), k));
    WL_CUDA(cudaMemcpyAsync(S.coef.p, SL.lam.data(), sizeof(double) * k, cudaMemcpyHostToDevice, S.s));
    k_scale_vec<<<WL_GRID(n2 * k, 256), 256, 0, S.s>>>(SL.tmp2.as<zd>(), SL.tmp2.as<zd>(), S.coef.as<double>(), n2 / 2, k, 1);
    WL_TRY(wl::stencil_apply(a, l, WL_FP64, V, SL.tmp1.p, SL.tmp2.p, k, S.s));
    WL_TRY(wl::kaczmarz_sweeps(a, l, WL_FP64, V, SL.tmp1.p, k, 1, S.s));
    WL_TRY(ritz(S, l, V, k, SL.lam, tn));
  }
  std::vector<double> lam2;
  WL_TRY(ritz(S, l, V, k, lam2, tn));
  std::vector<double> sc(k);
  for (int q = 0; q < k; ++q) sc[q] = tn[q] > 0 ? 1.0 / sqrt(tn[q]) : 0.0;
  WL_CUDA(cudaMemcpyAsync(S.coef.p, sc.data(), sizeof(double) * k, cudaMemcpyHostToDevice, S.s));
  k_scale_vec<<<WL_GRID(n2 * k, 256), 256, 0, S.s>>>(V, V, S.coef.as<double>(), n2 / 2, k, 0);
  WL_CUDA(cudaGetLastError());
  WL_CUDA(cudaStreamSynchronize(S.s));
  return WL_OK;
}

static int relax_both(Setup &S, int l, int mu, bool with_e) {
  WL_TRY(relax_homog(S, l, S.S[l].Vr.as<zd>(), S.kr, mu));
  if (with_e) WL_TRY(relax_eig(S, l, mu));
  return WL_OK;
}

// Sec. 3.3: LS fit with all test vectors of level l, then Galerkin (Sec. 3.5)
static int fit_level(Setup &S, int l) {
  wl_amg *a = S.a;
  SetupLevel &SL = S.S[l];
  Level &F = a->lev[l], &Cl = a->lev[l + 1];
  long n2 = n2of(a, l);
  int ke = SL.have_e ? S.ke : 0, k = S.kr + ke;
  std::vector<double> lr, tr, le, te;
  WL_TRY(ritz(S, l, SL.Vr.as<zd>(), S.kr, lr, tr));
  if (ke) WL_TRY(ritz(S, l, SL.Ve.as<zd>(), ke, le, te));
  std::vector<double> sc(k), w(k);
  for (int q = 0; q < k; ++q) {
    double t = q < S.kr ? tr[q] : te[q - S.kr];
    double lam = q < S.kr ? lr[q] : le[q - S.kr];
    sc[q] = t > 0 ? 1.0 / sqrt(t) : 0.0;
    w[q] = 1.0 / std::max(fabs(lam), 1e-12);  // reading of the weights of Eq. 3.4
  }
  WL_TRY(S.W.alloc(sizeof(zd) * n2 * k));
  WL_TRY(S.wts.alloc(sizeof(double) * 2 * 64));
  WL_CUDA(cudaMemcpyAsync(S.wts.p, sc.data(), sizeof(double) * k, cudaMemcpyHostToDevice, S.s));
  WL_CUDA(cudaMemcpyAsync(S.wts.as<double>() + 64, w.data(), sizeof(double) * k, cudaMemcpyHostToDevice, S.s));
  k_gather_tv<<<WL_GRID(n2 * k, 256), 256, 0, S.s>>>(SL.Vr.as<zd>(), S.kr, ke ? SL.Ve.as<zd>() : nullptr, ke,
                                                     S.wts.as<double>(), S.W.as<zd>(), n2);
  int lgB = ilog2(F.B);
  k_ls_fit<<<WL_GRID(2 * F.n, 128), 128, 0, S.s>>>(F.geo, Cl.geo, lgB, S.W.as<zd>(), S.wts.as<double>() + 64, k,
                                                   F.op64.P.as<zd>());
  k_galerkin<<<WL_GRID(Cl.n * 9, 64), 64, 0, S.s>>>(F.geo, Cl.geo, lgB, F.op64.A.as<zd>(), F.op64.P.as<zd>(),
                                                    Cl.op64.A.as<zd>());
  WL_TRY(wl::symmetrise_stencil(Cl.N, Cl.op64.A.as<zd>(), S.s));
  WL_TRY(wl::compute_den64(Cl.N, Cl.op64.A.as<zd>(), Cl.op64.den.as<double>(), S.s));
  const zd *Tf = S.S[l].T.as<zd>();
  k_galerkin<<<WL_GRID(Cl.n * 9, 64), 64, 0, S.s>>>(F.geo, Cl.geo, lgB, Tf, F.op64.P.as<zd>(), S.S[l + 1].T.as<zd>());
  k_herm_stencil<<<WL_GRID(Cl.n * 5, 128), 128, 0, S.s>>>(Cl.geo, S.S[l + 1].T.as<zd>());
  WL_CUDA(cudaGetLastError());
  WL_CUDA(cudaStreamSynchronize(S.s));
  return WL_OK;
}

static int inject_all(Setup &S, int l) {
  wl_amg *a = S.a;
  Level &F = a->lev[l], &Cl = a->lev[l + 1];
  int lgB = ilog2(F.B);
  k_inject<<<WL_GRID((long)Cl.n * S.kr, 256), 256, 0, S.s>>>(F.geo, Cl.geo, lgB, S.S[l].Vr.as<zd>(),
                                                            S.S[l + 1].Vr.as<zd>(), S.kr);
  if (S.S[l].have_e && S.ke) {
    k_inject<<<WL_GRID((long)Cl.n * S.ke, 256), 256, 0, S.s>>>(F.geo, Cl.geo, lgB, S.S[l].Ve.as<zd>(),
                                                              S.S[l + 1].Ve.as<zd>(), S.ke);
    S.S[l + 1].lam = S.S[l].lam;
    S.S[l + 1].have_e = true;
  }
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

static int interp_e(Setup &S, int l) {
  wl_amg *a = S.a;
  if (!S.ke) return WL_OK;
  long n2 = n2of(a, l);
  WL_CUDA(cudaMemsetAsync(S.S[l].Ve.p, 0, sizeof(zd) * n2 * S.ke, S.s));
  WL_TRY(wl::prolong_op(a, l, WL_FP64, S.S[l + 1].Ve.p, S.S[l].Ve.p, S.ke, S.s));
  S.S[l].lam = S.S[l + 1].lam;
  S.S[l].have_e = true;
  return WL_OK;
}

// Thm. 3.1 (i) on the coarsest grid: k_e eigenpairs of Z v = lambda T v with
// the smallest |lambda|, T-orthonormal
static int coarsest_eig(Setup &S) {
  wl_amg *a = S.a;
  int l = a->L - 1;
  Level &C = a->lev[l];
  int n = 2 * C.n;
  if (!S.ke) return WL_OK;
  DBuf Z, T, Wv, work, info, cols;
  WL_TRY(Z.alloc(sizeof(zd) * n * n));
  WL_TRY(T.alloc(sizeof(zd) * n * n));
  WL_TRY(Wv.alloc(sizeof(double) * n));
  WL_TRY(info.alloc(sizeof(int)));
  WL_CUDA(cudaMemsetAsync(Z.p, 0, sizeof(zd) * n * n, S.s));
  WL_CUDA(cudaMemsetAsync(T.p, 0, sizeof(zd) * n * n, S.s));
  k_stencil_dense_cm<<<WL_GRID(C.n, 128), 128, 0, S.s>>>(C.geo, C.op64.A.as<zd>(), Z.as<zd>(), 1);
  k_stencil_dense_cm<<<WL_GRID(C.n, 128), 128, 0, S.s>>>(C.geo, S.S[l].T.as<zd>(), T.as<zd>(), 0);
  WL_CUDA(cudaGetLastError());
  if (!S.cs) {
    if (cusolverDnCreate(&S.cs) != CUSOLVER_STATUS_SUCCESS) {
      wl_set_error("cusolverDnCreate failed");
      return WL_ECUDA;
    }
  }
  cusolverDnSetStream(S.cs, S.s);
  int lwork = 0;
  if (cusolverDnZhegvd_bufferSize(S.cs, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                  (cuDoubleComplex *)Z.p, n, (cuDoubleComplex *)T.p, n, Wv.as<double>(),
                                  &lwork) != CUSOLVER_STATUS_SUCCESS) {
    wl_set_error("zhegvd_bufferSize failed");
    return WL_ECUDA;
  }
  WL_TRY(work.alloc(sizeof(cuDoubleComplex) * (size_t)std::max(lwork, 1)));
  if (cusolverDnZhegvd(S.cs, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                       (cuDoubleComplex *)Z.p, n, (cuDoubleComplex *)T.p, n, Wv.as<double>(),
                       (cuDoubleComplex *)work.p, lwork, info.as<int>()) != CUSOLVER_STATUS_SUCCESS) {
    wl_set_error("zhegvd failed");
    return WL_ECUDA;
  }
  std::vector<double> lam(n);
  int hinfo = 0;
  WL_CUDA(cudaMemcpyAsync(lam.data(), Wv.p, sizeof(double) * n, cudaMemcpyDeviceToHost, S.s));
  WL_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, S.s));
  WL_CUDA(cudaStreamSynchronize(S.s));
  if (hinfo != 0) {
    wl_set_error("zhegvd info = %d (mass matrix not positive definite?)", hinfo);
    return WL_BAD_HIERARCHY;
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return fabs(lam[x]) < fabs(lam[y]); });
  std::vector<int> pick(ord.begin(), ord.begin() + S.ke);
  WL_TRY(cols.alloc(sizeof(int) * S.ke));
  WL_CUDA(cudaMemcpyAsync(cols.p, pick.data(), sizeof(int) * S.ke, cudaMemcpyHostToDevice, S.s));
  k_take_eigvecs<<<WL_GRID(n * S.ke, 256), 256, 0, S.s>>>(Z.as<zd>(), n, cols.as<int>(), S.ke, S.S[l].Ve.as<zd>());
  WL_CUDA(cudaGetLastError());
  S.S[l].lam.resize(S.ke);
  for (int q = 0; q < S.ke; ++q) S.S[l].lam[q] = lam[pick[q]];
  S.S[l].have_e = true;
  WL_CUDA(cudaStreamSynchronize(S.s));
  Z.release();
  T.release();
  Wv.release();
  work.release();
  info.release();
  cols.release();
  return WL_OK;
}

// Fig. 3.2: one W-visit of level l >= 1
static int visit(Setup &S, int l, bool first, int mu) {
  wl_amg *a = S.a;
  if (l == a->L - 1) return coarsest_eig(S);
  WL_TRY(relax_both(S, l, mu, !first));
  WL_TRY(fit_level(S, l));
  WL_TRY(inject_all(S, l));
  WL_TRY(visit(S, l + 1, first, mu));
  WL_TRY(interp_e(S, l));
  WL_TRY(relax_both(S, l, mu, true));
  WL_TRY(fit_level(S, l));
  WL_TRY(inject_all(S, l));
  WL_TRY(visit(S, l + 1, false, mu));
  WL_TRY(interp_e(S, l));
  return relax_eig(S, l, mu);
}

// Sec. 4.2 super-V setup: one visit per grid, mu 2^l relaxations before
// (both sets, then fit and injection) and after (eigenvector set) the
// coarse visit, so each grid relaxes as often as in the W-visits above while
// the coarsest eigensolve runs once per setup cycle
static int visit_superv(Setup &S, int l, bool first, int mu) {
  wl_amg *a = S.a;
  if (l == a->L - 1) return coarsest_eig(S);
  int mul = mu << l;
  WL_TRY(relax_both(S, l, mul, !first));
  WL_TRY(fit_level(S, l));
  WL_TRY(inject_all(S, l));
  WL_TRY(visit_superv(S, l + 1, first, mu));
  WL_TRY(interp_e(S, l));
  return relax_eig(S, l, mul);
}

__global__ void k_axpy_col(zd *V, const zd *e, long n2, int k, int q) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) V[i * k + q] = V[i * k + q] + e[i];
}
__global__ void k_get_col(const zd *V, zd *out, long n2, int k, int q, double sign) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) out[i] = sign * V[i * k + q];
}

// Sec. 4.1 adaptive step: two solver cycles on A_0 v = 0 for the finest-grid
// test vector with the smallest |lambda|
static int adaptive_step(Setup &S) {
  wl_amg *a = S.a;
  long n2 = n2of(a, 0);
  std::vector<double> lr, tr, le, te;
  WL_TRY(ritz(S, 0, S.S[0].Vr.as<zd>(), S.kr, lr, tr));
  if (S.S[0].have_e && S.ke) WL_TRY(ritz(S, 0, S.S[0].Ve.as<zd>(), S.ke, le, te));
  int best = -1;
  double bl = INFINITY;
  for (int q = 0; q < S.kr; ++q)
    if (fabs(lr[q]) < bl) bl = fabs(lr[q]), best = q;
  for (int q = 0; q < (int)le.size(); ++q)
    if (fabs(le[q]) < bl) bl = fabs(le[q]), best = S.kr + q;
  if (best < 0) return WL_OK;
  bool inE = best >= S.kr;
  zd *Vb = inE ? S.S[0].Ve.as<zd>() : S.S[0].Vr.as<zd>();
  int kb = inE ? S.ke : S.kr, qb = inE ? best - S.kr : best;
  WL_TRY(wl::coarsest_invert(a));
  WL_TRY(wl::ensure_workspace(a, 1, WL_FP64));
  amg_params save = a->prm;
  a->prm.nu_pre = 4;  // the paper's W(4,4) cycle
  a->prm.nu_post = 4;
  a->prm.cycle = WL_CYCLE_W;
  Level &L0 = a->lev[0];
  int rc = WL_OK;
  for (int it = 0; it < 2 && !rc; ++it) {
    k_get_col<<<WL_GRID(n2, 256), 256, 0, S.s>>>(Vb, S.S[0].tmp2.as<zd>(), n2, kb, qb, 1.0);
    rc = wl::stencil_apply(a, 0, WL_FP64, S.S[0].tmp2.p, L0.f.p, S.S[0].zero.p, 1, S.s);  // f = -A v
    if (!rc) rc = wl::cycle_direct(a, 1, WL_FP64, S.s);
    if (!rc) k_axpy_col<<<WL_GRID(n2, 256), 256, 0, S.s>>>(Vb, L0.x.as<zd>(), n2, kb, qb);
  }
  a->prm = save;
  WL_TRY(rc);
  // T-normalise the updated vector (T_0 = I) and refresh its Ritz value
  if (inE) {
    std::vector<double> l2, t2;
    WL_TRY(ritz(S, 0, S.S[0].Ve.as<zd>(), S.ke, l2, t2));
    S.S[0].lam[qb] = l2[qb];
  }
  WL_CUDA(cudaStreamSynchronize(S.s));
  return WL_OK;
}

}  // namespace

extern "C" int amg_setup(wl_op *op, const amg_params *params, wl_amg **out) {
  if (!op || !out) {
    wl_set_error("amg_setup: invalid argument");
    return WL_EINVAL;
  }
  *out = nullptr;
  amg_params prm;
  if (params) prm = *params;
  else amg_params_default(&prm);
  int Nl[8];
  WL_TRY(wl::resolve_levels(op->N, &prm, Nl));
  if (prm.k_r < 1 || prm.k_e < 0 || prm.k_r + prm.k_e > 64 || prm.setup_mu[0] < 0 || prm.setup_mu[1] < 0) {
    wl_set_error("amg_setup: need 1 <= k_r, 0 <= k_e, k_r + k_e <= 64");
    return WL_EINVAL;
  }
  WL_TRY(wl::enter(op));
  wl_amg *a = new wl_amg();
  a->op = op;
  wl::op_retain(op);
  a->prm = prm;
  // the setup relaxes with the 16-colour ordering of Sec. 3.1 whatever
  // ordering the solve phase uses (kacz_order is restored below)
  a->prm.kacz_order = 0;
  a->L = prm.levels;
  a->cap = 0;
  a->h_small = nullptr;
  Setup S;
  S.a = a;
  S.kr = prm.k_r;
  S.ke = prm.k_e;
  S.s = op->stream;
  int rc = wl::hier_alloc(a, Nl);
  for (int l = 0; l < a->L && !rc; ++l) {
    long n2 = (long)a->lev[l].n * 2;
    int kmax = std::max(S.kr, std::max(S.ke, 1));
    rc = S.S[l].Vr.alloc(sizeof(zd) * n2 * S.kr);
    if (!rc) rc = S.S[l].Ve.alloc(sizeof(zd) * n2 * std::max(S.ke, 1));
    if (!rc) rc = S.S[l].T.alloc(sizeof(zd) * (size_t)a->lev[l].n * 36);
    if (!rc) rc = S.S[l].tmp1.alloc(sizeof(zd) * n2 * kmax);
    if (!rc) rc = S.S[l].tmp2.alloc(sizeof(zd) * n2 * kmax);
    if (!rc) rc = S.S[l].zero.alloc(sizeof(zd) * n2 * kmax);
    if (!rc && cudaMemsetAsync(S.S[l].zero.p, 0, sizeof(zd) * n2 * kmax, S.s) != cudaSuccess) rc = WL_ECUDA;
    if (!rc) rc = a->lev[l].op64.den.alloc(sizeof(double) * a->lev[l].n * 2);
  }
  if (!rc) {
    k_identity_stencil<<<WL_GRID((long)a->lev[0].n * 36, 256), 256, 0, S.s>>>(a->lev[0].n, S.S[0].T.as<zd>());
    rc = wl::build_dhat_stencil(op, a->lev[0].op64.A.as<zd>(), S.s);
  }
  if (!rc) rc = wl::compute_den64(a->lev[0].N, a->lev[0].op64.A.as<zd>(), a->lev[0].op64.den.as<double>(), S.s);
  if (!rc) {
    long n2 = (long)a->lev[0].n * 2;
    k_random_vectors<<<WL_GRID(n2 * S.kr, 256), 256, 0, S.s>>>(n2, S.kr, prm.seed, S.S[0].Vr.as<zd>());
    if (cudaGetLastError() != cudaSuccess) rc = WL_ECUDA;
  }
  // setup cycle 1
  if (!rc) rc = relax_both(S, 0, prm.setup_mu[0], false);
  if (!rc) rc = fit_level(S, 0);
  if (!rc) rc = inject_all(S, 0);
  if (!rc) rc = prm.setup_cycle == 1 ? visit_superv(S, 1, true, prm.setup_mu[0]) : visit(S, 1, true, prm.setup_mu[0]);
  if (!rc) rc = interp_e(S, 0);
  if (!rc) rc = adaptive_step(S);
  // setup cycle 2
  if (!rc) rc = relax_both(S, 0, prm.setup_mu[1], true);
  if (!rc) rc = fit_level(S, 0);
  if (!rc) rc = inject_all(S, 0);
  if (!rc) rc = prm.setup_cycle == 1 ? visit_superv(S, 1, false, prm.setup_mu[1])
                                     : visit(S, 1, false, prm.setup_mu[1]);
  if (!rc) rc = interp_e(S, 0);
  a->prm.kacz_order = prm.kacz_order;
  if (!rc) rc = wl::hier_finish(a);
  if (S.cs) cusolverDnDestroy(S.cs);
  cudaStreamSynchronize(S.s);
  for (int l = 0; l < 8; ++l) {
    S.S[l].Vr.release();
    S.S[l].Ve.release();
    S.S[l].T.release();
    S.S[l].tmp1.release();
    S.S[l].tmp2.release();
    S.S[l].zero.release();
  }
  S.red.release();
  S.coef.release();
  S.W.release();
  S.wts.release();
  if (rc) {
    wl::amg_free(a);
    return rc;
  }
  *out = a;
  return WL_OK;
}
