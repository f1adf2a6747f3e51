// wl_ops.cu -- the Wilson operator on the GPU: folded links, matrix-free
// Dhat (Sec. 3.2, Eq. 3.2) and D (Sec. 2, Eq. 2.1), the two-step Schur
// reduction / reconstruction, the explicit Dhat stencil used by the cycle,
// layout conversions, and the error state of the C ABI.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "wl_common.cuh"

// ------------------------------------------------------------ error state
static thread_local char g_err[512];

void wl_set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char *wl_last_error(void) { return g_err; }

#include <atomic>
static std::atomic<long long> g_launches(0);
void wl_count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
extern "C" long long wl_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int DBuf::alloc(size_t b) {
  if (b <= bytes && p) return WL_OK;
  if (!own) {
    wl_set_error("internal: a borrowed buffer of %zu bytes cannot grow to %zu", bytes, b);
    return WL_EINVAL;
  }
  release();
  if (b == 0) return WL_OK;
  cudaError_t e = cudaMalloc(&p, b);
  if (e != cudaSuccess) {
    p = nullptr;
    bytes = 0;
    cudaGetLastError();
    wl_set_error("cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
    return WL_OOM;
  }
  bytes = b;
  return WL_OK;
}

void DBuf::release() {
  if (p && own) cudaFree(p);
  p = nullptr;
  bytes = 0;
  own = true;
}

// ------------------------------------------------------------- hop algebra
// K_{p, p+mu} v = (1 - s_mu) V_mu(p) v,  K_{p, p-mu} v = (1 + s_mu) conj(V_mu(p-mu)) v
// with the spin projections (1 -+ s_1) v = (w, -+w), w = v0 -+ v1 and
// (1 -+ s_2) v = (w, -+i w), w = v0 +- i v1 (s_2 = [[0,-i],[i,0]]).
template <typename T>
__device__ __forceinline__ void hop_acc(cx<T> &o0, cx<T> &o1, int mu, int fwd, cx<T> link,
                                        cx<T> v0, cx<T> v1) {
  cx<T> w;
  if (mu == 0) w = fwd ? v0 - v1 : v0 + v1;
  else w = fwd ? v0 + ci(v1) : v0 - ci(v1);
  w = (fwd ? link : cconj(link)) * w;
  o0 = o0 + w;
  if (mu == 0) o1 = fwd ? o1 - w : o1 + w;
  else o1 = fwd ? o1 - ci(w) : o1 + ci(w);
}

// folded links: V_mu(x,y) = U_mu(x,y) / (2c), times -1 on y-links leaving y = N-1
__global__ void k_fold_links(int N, double kappa, const zd *U, zd *V64, zf *V32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * N * N) return;
  int mu = i / (N * N), y = (i / N) % N;
  double s = (mu == 1 && y == N - 1) ? -kappa : kappa;
  zd u = U[i];
  zd v = mk(s * u.re, s * u.im);
  V64[i] = v;
  V32[i] = ccast<float>(v);
}

// out(site of parity par_out) = sum of the four hops of K applied to `in`
// (sites of the other parity); if sub != nullptr: out = sub - K in.
// Layout of in/out/sub: [h][2][nrhs] over the half lattice.
template <typename Tc, typename Tin, typename Tsub, typename Tout>
__global__ void k_hop(Geo g, const cx<Tc> *__restrict__ V, int par_out,
                      const cx<Tin> *__restrict__ in, const cx<Tsub> *__restrict__ sub,
                      cx<Tout> *__restrict__ out, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int n = g.nsites();
  if (tid >= (long)n * nrhs) return;
  int h = (int)(tid / nrhs), r = (int)(tid - (long)h * nrhs);
  int y = h >> (g.lg - 1);
  int x = ((h & (g.half() - 1)) << 1) | ((y + par_out) & 1);
  int N = g.N;
  cx<Tc> o0 = mk<Tc>(0, 0), o1 = mk<Tc>(0, 0);
#pragma unroll
  for (int mu = 0; mu < 2; ++mu) {
#pragma unroll
    for (int fwd = 1; fwd >= 0; --fwd) {
      int dx = (mu == 0) ? (fwd ? 1 : -1) : 0, dy = (mu == 1) ? (fwd ? 1 : -1) : 0;
      int xn = (x + dx) & (N - 1), yn = (y + dy) & (N - 1);
      int lx = fwd ? x : xn, ly = fwd ? y : yn;  // link V_mu(p) or V_mu(p - mu)
      cx<Tc> link = V[(mu * N + ly) * N + lx];
      long j = (long)g.idx(xn, yn) * 2 * nrhs + r;
      cx<Tc> v0 = widen<Tc>(in[j]), v1 = widen<Tc>(in[j + nrhs]);
      hop_acc(o0, o1, mu, fwd, link, v0, v1);
    }
  }
  long o = (long)h * 2 * nrhs + r;
  if (sub) {
    o0 = widen<Tc>(sub[o]) - o0;
    o1 = widen<Tc>(sub[o + nrhs]) - o1;
  }
  out[o] = ccast<Tout>(o0);
  out[o + nrhs] = ccast<Tout>(o1);
}

// D psi on the full lattice, ABI layout [nrhs][N][N][2]: D = c (I - K);
// g5 = 1 gives Z psi = Gamma5 D psi (Thm. 3.1: the spin-1 row negated, an
// exact sign flip of the D result)
template <typename Tc>
__global__ void k_wilson_full(int N, double c, const cx<Tc> *__restrict__ V,
                              const zd *__restrict__ in, zd *__restrict__ out, int nrhs, int g5) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long nz = (long)N * N;
  if (tid >= nz * nrhs) return;
  int r = (int)(tid / nz);
  int z = (int)(tid - (long)r * nz);
  int y = z / N, x = z % N;
  const zd *b = in + (long)r * nz * 2;
  cx<Tc> o0 = mk<Tc>(0, 0), o1 = mk<Tc>(0, 0);
  for (int mu = 0; mu < 2; ++mu)
    for (int fwd = 1; fwd >= 0; --fwd) {
      int dx = (mu == 0) ? (fwd ? 1 : -1) : 0, dy = (mu == 1) ? (fwd ? 1 : -1) : 0;
      int xn = (x + dx) & (N - 1), yn = (y + dy) & (N - 1);
      int lx = fwd ? x : xn, ly = fwd ? y : yn;
      cx<Tc> link = V[(mu * N + ly) * N + lx];
      long j = ((long)yn * N + xn) * 2;
      hop_acc(o0, o1, mu, fwd, link, ccast<Tc>(b[j]), ccast<Tc>(b[j + 1]));
    }
  long o = ((long)r * nz + z) * 2;
  cx<Tc> p0 = ccast<Tc>(in[o]), p1 = ccast<Tc>(in[o + 1]);
  Tc cc = (Tc)c;
  out[o] = ccast<double>(cc * (p0 - o0));
  out[o + 1] = ccast<double>((g5 ? -cc : cc) * (p1 - o1));
}

// bhat_e = b_e/c + K_eo (b_o/c); b in ABI layout [nrhs][N][N][2], bhat
// internal [n][2][nrhs] (FP64)
__global__ void k_eo_reduce(Geo g, double c, const zd *__restrict__ V, const zd *__restrict__ b,
                            zd *__restrict__ bh, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int n = g.nsites(), N = g.N;
  if (tid >= (long)n * nrhs) return;
  int h = (int)(tid / nrhs), r = (int)(tid - (long)h * nrhs);
  int x, y;
  g.xy(h, x, y);
  const zd *br = b + (long)r * N * N * 2;
  double ic = 1.0 / c;
  zd o0 = mk(0.0, 0.0), o1 = mk(0.0, 0.0);
  for (int mu = 0; mu < 2; ++mu)
    for (int fwd = 1; fwd >= 0; --fwd) {
      int dx = (mu == 0) ? (fwd ? 1 : -1) : 0, dy = (mu == 1) ? (fwd ? 1 : -1) : 0;
      int xn = (x + dx) & (N - 1), yn = (y + dy) & (N - 1);
      int lx = fwd ? x : xn, ly = fwd ? y : yn;
      zd link = V[(mu * N + ly) * N + lx];
      long j = ((long)yn * N + xn) * 2;
      hop_acc(o0, o1, mu, fwd, link, ic * br[j], ic * br[j + 1]);
    }
  long e = ((long)y * N + x) * 2;
  long o = (long)h * 2 * nrhs + r;
  bh[o] = ic * br[e] + o0;
  bh[o + nrhs] = ic * br[e + 1] + o1;
}

// psi_e = x_e, psi_o = b_o/c + K_oe x_e; psi, b in ABI layout, xe internal
__global__ void k_eo_reconstruct(Geo g, double c, const zd *__restrict__ V,
                                 const zd *__restrict__ b, const zd *__restrict__ xe,
                                 zd *__restrict__ psi, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int N = g.N;
  long nz = (long)N * N;
  if (tid >= nz * nrhs) return;
  int r = (int)(tid / nz);
  int z = (int)(tid - (long)r * nz);
  int y = z / N, x = z % N;
  long o = ((long)r * nz + z) * 2;
  if (((x + y) & 1) == 0) {
    long j = (long)g.idx(x, y) * 2 * nrhs + r;
    psi[o] = xe[j];
    psi[o + 1] = xe[j + nrhs];
    return;
  }
  zd o0 = mk(0.0, 0.0), o1 = mk(0.0, 0.0);
  for (int mu = 0; mu < 2; ++mu)
    for (int fwd = 1; fwd >= 0; --fwd) {
      int dx = (mu == 0) ? (fwd ? 1 : -1) : 0, dy = (mu == 1) ? (fwd ? 1 : -1) : 0;
      int xn = (x + dx) & (N - 1), yn = (y + dy) & (N - 1);
      int lx = fwd ? x : xn, ly = fwd ? y : yn;
      zd link = V[(mu * N + ly) * N + lx];
      long j = (long)g.idx(xn, yn) * 2 * nrhs + r;
      hop_acc(o0, o1, mu, fwd, link, xe[j], xe[j + nrhs]);
    }
  double ic = 1.0 / c;
  const zd *br = b + (long)r * nz * 2;
  psi[o] = ic * br[z * 2] + o0;
  psi[o + 1] = ic * br[z * 2 + 1] + o1;
}

// --------------------------------------------------- explicit Dhat stencil
struct M2 {
  zd a[2][2];
};
__device__ __forceinline__ M2 hopmat(int mu, int fwd, zd link) {
  // (1 - s_mu) V  (forward) or (1 + s_mu) conj(V) (backward)
  zd l = fwd ? link : cconj(link);
  double sg = fwd ? -1.0 : 1.0;
  M2 m;
  m.a[0][0] = l;
  m.a[1][1] = l;
  if (mu == 0) {
    m.a[0][1] = sg * l;
    m.a[1][0] = sg * l;
  } else {  // s_2 = [[0,-i],[i,0]]: +-s_2 has (0,1) = -+i, (1,0) = +-i
    m.a[0][1] = ci(mk(-sg * l.re, -sg * l.im));
    m.a[1][0] = ci(mk(sg * l.re, sg * l.im));
  }
  return m;
}
__device__ __forceinline__ M2 mmul(const M2 &p, const M2 &q) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.a[i][j] = p.a[i][0] * q.a[0][j] + p.a[i][1] * q.a[1][j];
  return r;
}
__device__ __forceinline__ zd link_of(const zd *V, int N, int x, int y, int mu, int fwd) {
  if (!fwd) {
    if (mu == 0) x = (x - 1) & (N - 1);
    else y = (y - 1) & (N - 1);
  }
  return V[(mu * N + y) * N + x];
}

// A[h][d][s][t] = Dhat_{(h,s),(nb(h,d),t)} = delta - sum over two-hop paths
__global__ void k_build_dhat(Geo g, const zd *__restrict__ V, zd *__restrict__ A) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.nsites()) return;
  int x, y, N = g.N;
  g.xy(h, x, y);
  for (int d = 0; d < 9; ++d) {
    int da = d / 3 - 1, db = d % 3 - 1;
    int dx = da + db, dy = da - db;
    M2 s;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) s.a[i][j] = mk(0.0, 0.0);
    if (dx == 0 && dy == 0) {
      // the four paths out and back cancel: (1 - s)(1 + s) = 0
    } else if (dy == 0 || dx == 0) {
      int mu = (dy == 0) ? 0 : 1, fwd = (dx + dy) > 0;
      int ox = x + (mu == 0 ? (fwd ? 1 : -1) : 0), oy = y + (mu == 1 ? (fwd ? 1 : -1) : 0);
      ox &= N - 1;
      oy &= N - 1;
      s = mmul(hopmat(mu, fwd, link_of(V, N, x, y, mu, fwd)),
               hopmat(mu, fwd, link_of(V, N, ox, oy, mu, fwd)));
    } else {
      int fx = dx > 0, fy = dy > 0;
      int o1x = (x + (fx ? 1 : -1)) & (N - 1), o1y = y;
      int o2x = x, o2y = (y + (fy ? 1 : -1)) & (N - 1);
      M2 p1 = mmul(hopmat(0, fx, link_of(V, N, x, y, 0, fx)),
                   hopmat(1, fy, link_of(V, N, o1x, o1y, 1, fy)));
      M2 p2 = mmul(hopmat(1, fy, link_of(V, N, x, y, 1, fy)),
                   hopmat(0, fx, link_of(V, N, o2x, o2y, 0, fx)));
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) s.a[i][j] = p1.a[i][j] + p2.a[i][j];
    }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        zd v = mk(-s.a[i][j].re, -s.a[i][j].im);
        if (d == 4 && i == j) v = mk(1.0, 0.0);
        if (d == 4 && i != j) v = mk(0.0, 0.0);
        A[((long)h * 9 + d) * 4 + i * 2 + j] = v;
      }
  }
}

// gamma5-Hermitian part: the pair (h, d) / (nb(h,d), 8-d) is averaged as
// X = (A_hd + g5 A_j,8-d^H g5) / 2, written to both slots; the centre block
// becomes (A + g5 A^H g5) / 2.  (g5 Y^H g5)_st = g_s g_t conj(Y_ts).
__global__ void k_symmetrise(Geo g, zd *A) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int n = g.nsites();
  if (tid >= n * 5) return;
  int h = tid / 5, q = tid % 5;
  int x, y;
  g.xy(h, x, y);
  const double gs[2] = {1.0, -1.0};
  if (q == 4) {
    zd *B = A + ((long)h * 9 + 4) * 4;
    zd b[2][2];
    for (int s = 0; s < 2; ++s)
      for (int t = 0; t < 2; ++t) b[s][t] = B[s * 2 + t];
    for (int s = 0; s < 2; ++s)
      for (int t = 0; t < 2; ++t) {
        zd m = cconj(b[t][s]);
        double f = gs[s] * gs[t];
        B[s * 2 + t] = mk(0.5 * (b[s][t].re + f * m.re), 0.5 * (b[s][t].im + f * m.im));
      }
    return;
  }
  int d = 5 + q;
  int j = g.nb(x, y, d);
  zd *B1 = A + ((long)h * 9 + d) * 4;
  zd *B2 = A + ((long)j * 9 + (8 - d)) * 4;
  zd b1[2][2], b2[2][2], X[2][2];
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) {
      b1[s][t] = B1[s * 2 + t];
      b2[s][t] = B2[s * 2 + t];
    }
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) {
      zd m = cconj(b2[t][s]);
      double f = gs[s] * gs[t];
      X[s][t] = mk(0.5 * (b1[s][t].re + f * m.re), 0.5 * (b1[s][t].im + f * m.im));
    }
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) {
      B1[s * 2 + t] = X[s][t];
      zd m = cconj(X[t][s]);
      double f = gs[s] * gs[t];
      B2[s * 2 + t] = mk(f * m.re, f * m.im);
    }
}

// den[h][t] = sum_{d,s} |A[h][d][t][s]|^2 (= ||A e_(h,t)||^2 for a
// gamma5-Hermitian A)
__global__ void k_den64(int n, const zd *__restrict__ A, double *__restrict__ den) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * n) return;
  int h = tid >> 1, t = tid & 1;
  double s = 0;
  for (int d = 0; d < 9; ++d)
    for (int u = 0; u < 2; ++u) s += cnorm2(A[((long)h * 9 + d) * 4 + t * 2 + u]);
  den[tid] = s;
}

// ABI [nrhs][n2] (FP64) <-> internal [n2][nrhs] in double or float
template <typename To>
__global__ void k_to_internal(const zd *__restrict__ src, cx<To> *__restrict__ dst, long n2,
                              int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n2 * nrhs) return;
  long i = tid / nrhs;
  int r = (int)(tid - i * nrhs);
  dst[tid] = ccast<To>(src[(long)r * n2 + i]);
}
template <typename Ti>
__global__ void k_from_internal(const cx<Ti> *__restrict__ src, zd *__restrict__ dst, long n2,
                                int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n2 * nrhs) return;
  int r = (int)(tid / n2);
  long i = tid - (long)r * n2;
  dst[tid] = ccast<double>(src[i * nrhs + r]);
}

namespace wl {

size_t prec_bytes(int prec) { return prec == WL_FP64 ? sizeof(zd) : sizeof(zf); }

int to_internal(const zd *src, void *dst, int n2, int nrhs, int prec, cudaStream_t s) {
  long tot = (long)n2 * nrhs;
  wl_count_launches(1);
  if (prec == WL_FP64) k_to_internal<double><<<WL_GRID(tot, 256), 256, 0, s>>>(src, (zd *)dst, n2, nrhs);
  else k_to_internal<float><<<WL_GRID(tot, 256), 256, 0, s>>>(src, (zf *)dst, n2, nrhs);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

int from_internal(const void *src, zd *dst, int n2, int nrhs, int prec, cudaStream_t s) {
  long tot = (long)n2 * nrhs;
  wl_count_launches(1);
  if (prec == WL_FP64) k_from_internal<double><<<WL_GRID(tot, 256), 256, 0, s>>>((const zd *)src, dst, n2, nrhs);
  else k_from_internal<float><<<WL_GRID(tot, 256), 256, 0, s>>>((const zf *)src, dst, n2, nrhs);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

// y = Dhat x (FP64 arithmetic, matrix-free, two hop kernels); x internal
// layout in double or float, y double.  Uses op->scratch for the odd field.
int dhat_apply_dev(wl_op *op, const void *x, int x_is_f32, zd *y, int nrhs, cudaStream_t s) {
  Geo g = op->geo;
  long n = g.nsites();
  WL_TRY(op->scratch.alloc(sizeof(zd) * n * 2 * nrhs));
  zd *t = op->scratch.as<zd>();
  unsigned grid = WL_GRID(n * nrhs, 256);
  const zd *V = op->Uf64.as<zd>();
  wl_count_launches(2);
  if (x_is_f32) {
    k_hop<double, float, double, double><<<grid, 256, 0, s>>>(g, V, 1, (const zf *)x, nullptr, t, nrhs);
    k_hop<double, double, float, double><<<grid, 256, 0, s>>>(g, V, 0, t, (const zf *)x, y, nrhs);
  } else {
    k_hop<double, double, double, double><<<grid, 256, 0, s>>>(g, V, 1, (const zd *)x, nullptr, t, nrhs);
    k_hop<double, double, double, double><<<grid, 256, 0, s>>>(g, V, 0, t, (const zd *)x, y, nrhs);
  }
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

int build_dhat_stencil(wl_op *op, zd *A, cudaStream_t s) {
  Geo g = op->geo;
  k_build_dhat<<<WL_GRID(g.nsites(), 128), 128, 0, s>>>(g, op->Uf64.as<zd>(), A);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return symmetrise_stencil(g.N, A, s);
}

int symmetrise_stencil(int N, zd *A, cudaStream_t s) {
  Geo g = make_geo(N);
  k_symmetrise<<<WL_GRID(g.nsites() * 5, 128), 128, 0, s>>>(g, A);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

int compute_den64(int N, const zd *A, double *den, cudaStream_t s) {
  int n = N * N / 2;
  k_den64<<<WL_GRID(2 * n, 256), 256, 0, s>>>(n, A, den);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

}  // namespace wl

// -------------------------------------------------------------- C ABI
// FNV-1a, 64 bit: offset basis 14695981039346656037, prime 1099511628211
static uint64_t fnv1a(const void *p, size_t n, uint64_t h = 14695981039346656037ULL) {
  const unsigned char *c = (const unsigned char *)p;
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ULL;
  return h;
}

static bool pow2_ge16(int L) { return L >= 16 && (L & (L - 1)) == 0; }

extern "C" int wilson_create(const void *gauge, int L, double m, void *cuda_stream, wl_op **out) {
  if (!out || !gauge) {
    wl_set_error("wilson_create: NULL argument");
    return WL_EINVAL;
  }
  *out = nullptr;
  if (!pow2_ge16(L)) {
    wl_set_error("wilson_create: L = %d must be a power of two >= 16", L);
    return WL_EINVAL;
  }
  if (m + 2.0 == 0.0) {
    wl_set_error("wilson_create: m + 2 must be non-zero");
    return WL_EINVAL;
  }
  wl_op *op = new wl_op();
  op->N = L;
  op->m = m;
  op->c = m + 2.0;
  op->user = (cudaStream_t)cuda_stream;
  op->geo = make_geo(L);
  cudaGetDevice(&op->device);
  if (cudaStreamCreateWithFlags(&op->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&op->ev, cudaEventDisableTiming) != cudaSuccess) {
    wl_set_error("wilson_create: cannot create the work stream");
    delete op;
    return WL_ECUDA;
  }
  if (wl::enter(op)) {
    wl_destroy(op);
    return WL_ECUDA;
  }
  size_t nl = (size_t)2 * L * L;
  DBuf tmp;
  int rc = tmp.alloc(sizeof(zd) * nl);
  if (!rc) rc = op->Uf64.alloc(sizeof(zd) * nl);
  if (!rc) rc = op->Uf32.alloc(sizeof(zf) * nl);
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(tmp.p, gauge, sizeof(zd) * nl, cudaMemcpyDefault, op->stream);
    if (e == cudaSuccess) {
      k_fold_links<<<WL_GRID(nl, 256), 256, 0, op->stream>>>(L, 1.0 / (2.0 * op->c), tmp.as<zd>(),
                                                              op->Uf64.as<zd>(), op->Uf32.as<zf>());
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      std::vector<zd> h(nl);
      e = cudaMemcpyAsync(h.data(), tmp.p, sizeof(zd) * nl, cudaMemcpyDeviceToHost, op->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(op->stream);
      op->gauge_hash = fnv1a(h.data(), sizeof(zd) * nl);
    }
    if (e != cudaSuccess) {
      wl_set_error("wilson_create: %s", cudaGetErrorString(e));
      rc = WL_ECUDA;
    }
  }
  tmp.release();
  if (rc) {
    wl_destroy(op);
    return rc;
  }
  *out = op;
  return WL_OK;
}

static void op_free(wl_op *op) {
  if (op->stream) cudaStreamSynchronize(op->stream);
  op->Uf64.release();
  op->Uf32.release();
  op->scratch.release();
  if (op->ev) cudaEventDestroy(op->ev);
  if (op->stream) cudaStreamDestroy(op->stream);
  delete op;
}

extern "C" void wl_destroy(wl_op *op) {
  if (op) wl::op_release(op);
}

namespace wl {
void op_retain(wl_op *op) { op->refs.fetch_add(1); }
void op_release(wl_op *op) {
  if (op->refs.fetch_sub(1) == 1) op_free(op);
}
}  // namespace wl

namespace wl {
int enter(wl_op *op) {
  WL_CUDA(cudaEventRecord(op->ev, op->user));
  WL_CUDA(cudaStreamWaitEvent(op->stream, op->ev, 0));
  return WL_OK;
}
}  // namespace wl

extern "C" int wl_apply(wl_op *op, int which, const void *x, void *y, int nrhs, int prec) {
  if (!op || !x || !y || nrhs < 1 || (prec != WL_FP64 && prec != WL_FP32) ||
      (which != WL_OP_D && which != WL_OP_DHAT && which != WL_OP_Z)) {
    wl_set_error("wl_apply: invalid argument");
    return WL_EINVAL;
  }
  WL_TRY(wl::enter(op));
  cudaStream_t s = op->stream;
  Geo g = op->geo;
  int N = op->N;
  if (which == WL_OP_D || which == WL_OP_Z) {
    long tot = (long)N * N * nrhs;
    int g5 = which == WL_OP_Z;
    if (prec == WL_FP64)
      k_wilson_full<double><<<WL_GRID(tot, 256), 256, 0, s>>>(N, op->c, op->Uf64.as<zd>(), (const zd *)x, (zd *)y,
                                                              nrhs, g5);
    else
      k_wilson_full<float><<<WL_GRID(tot, 256), 256, 0, s>>>(N, op->c, op->Uf32.as<zf>(), (const zd *)x, (zd *)y,
                                                             nrhs, g5);
    WL_CUDA(cudaGetLastError());
    return WL_OK;
  }
  long n = g.nsites();
  size_t eb = prec == WL_FP64 ? sizeof(zd) : sizeof(zf);
  DBuf xi, yi, t;
  int rc = xi.alloc(eb * n * 2 * nrhs);
  if (!rc) rc = yi.alloc(eb * n * 2 * nrhs);
  if (!rc) rc = t.alloc(eb * n * 2 * nrhs);
  if (!rc) rc = wl::to_internal((const zd *)x, xi.p, (int)(2 * n), nrhs, prec, s);
  if (!rc) {
    unsigned grid = WL_GRID(n * nrhs, 256);
    if (prec == WL_FP64) {
      const zd *V = op->Uf64.as<zd>();
      k_hop<double, double, double, double><<<grid, 256, 0, s>>>(g, V, 1, xi.as<zd>(), nullptr, t.as<zd>(), nrhs);
      k_hop<double, double, double, double><<<grid, 256, 0, s>>>(g, V, 0, t.as<zd>(), xi.as<zd>(), yi.as<zd>(), nrhs);
    } else {
      const zf *V = op->Uf32.as<zf>();
      k_hop<float, float, float, float><<<grid, 256, 0, s>>>(g, V, 1, xi.as<zf>(), nullptr, t.as<zf>(), nrhs);
      k_hop<float, float, float, float><<<grid, 256, 0, s>>>(g, V, 0, t.as<zf>(), xi.as<zf>(), yi.as<zf>(), nrhs);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      wl_set_error("wl_apply: %s", cudaGetErrorString(e));
      rc = WL_ECUDA;
    }
  }
  if (!rc) rc = wl::from_internal(yi.p, (zd *)y, (int)(2 * n), nrhs, prec, s);
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      wl_set_error("wl_apply: %s", cudaGetErrorString(e));
      rc = WL_ECUDA;
    }
  }
  xi.release();
  yi.release();
  t.release();
  return rc;
}

extern "C" int wl_eo_reduce(wl_op *op, const void *b, void *bhat, int nrhs) {
  if (!op || !b || !bhat || nrhs < 1) {
    wl_set_error("wl_eo_reduce: invalid argument");
    return WL_EINVAL;
  }
  WL_TRY(wl::enter(op));
  Geo g = op->geo;
  long n = g.nsites();
  DBuf t;
  WL_TRY(t.alloc(sizeof(zd) * n * 2 * nrhs));
  k_eo_reduce<<<WL_GRID(n * nrhs, 256), 256, 0, op->stream>>>(g, op->c, op->Uf64.as<zd>(), (const zd *)b, t.as<zd>(), nrhs);
  int rc = WL_OK;
  if (cudaGetLastError() != cudaSuccess) rc = WL_ECUDA;
  if (!rc) rc = wl::from_internal(t.p, (zd *)bhat, (int)(2 * n), nrhs, WL_FP64, op->stream);
  cudaStreamSynchronize(op->stream);
  t.release();
  return rc;
}

extern "C" int wl_eo_reconstruct(wl_op *op, const void *b, const void *xe, void *psi, int nrhs) {
  if (!op || !b || !xe || !psi || nrhs < 1) {
    wl_set_error("wl_eo_reconstruct: invalid argument");
    return WL_EINVAL;
  }
  WL_TRY(wl::enter(op));
  Geo g = op->geo;
  long n = g.nsites();
  DBuf t;
  WL_TRY(t.alloc(sizeof(zd) * n * 2 * nrhs));
  int rc = wl::to_internal((const zd *)xe, t.p, (int)(2 * n), nrhs, WL_FP64, op->stream);
  long tot = (long)op->N * op->N * nrhs;
  if (!rc) {
    k_eo_reconstruct<<<WL_GRID(tot, 256), 256, 0, op->stream>>>(g, op->c, op->Uf64.as<zd>(), (const zd *)b, t.as<zd>(), (zd *)psi, nrhs);
    if (cudaGetLastError() != cudaSuccess) rc = WL_ECUDA;
  }
  cudaStreamSynchronize(op->stream);
  t.release();
  return rc;
}

// used by amg_solve: reduce / reconstruct straight into / from the internal
// FP64 layout
namespace wl {
int eo_reduce_internal(wl_op *op, const zd *b, zd *bh, int nrhs, cudaStream_t s) {
  Geo g = op->geo;
  long n = g.nsites();
  k_eo_reduce<<<WL_GRID(n * nrhs, 256), 256, 0, s>>>(g, op->c, op->Uf64.as<zd>(), b, bh, nrhs);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}
int eo_reconstruct_internal(wl_op *op, const zd *b, const zd *xe, zd *psi, int nrhs, cudaStream_t s) {
  Geo g = op->geo;
  long tot = (long)op->N * op->N * nrhs;
  k_eo_reconstruct<<<WL_GRID(tot, 256), 256, 0, s>>>(g, op->c, op->Uf64.as<zd>(), b, xe, psi, nrhs);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}
// guess for x from a full field: x_e of psi in internal layout
__global__ void k_take_even(Geo g, const zd *__restrict__ psi, zd *__restrict__ xe, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int n = g.nsites(), N = g.N;
  if (tid >= (long)n * nrhs) return;
  int h = (int)(tid / nrhs), r = (int)(tid - (long)h * nrhs);
  int x, y;
  g.xy(h, x, y);
  long src = (((long)r * N + y) * N + x) * 2;
  long o = (long)h * 2 * nrhs + r;
  xe[o] = psi[src];
  xe[o + nrhs] = psi[src + 1];
}
int take_even_internal(wl_op *op, const zd *psi, zd *xe, int nrhs, cudaStream_t s) {
  Geo g = op->geo;
  long n = g.nsites();
  k_take_even<<<WL_GRID(n * nrhs, 256), 256, 0, s>>>(g, psi, xe, nrhs);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}
uint64_t hash_bytes(const void *p, size_t n) { return fnv1a(p, n); }
}  // namespace wl

extern "C" unsigned long long wl_hash_bytes(const void *p, size_t n) { return p || !n ? fnv1a(p, n) : 0ULL; }
