// wl_common.cuh -- internal types, complex helpers, lattice geometry and the
// host-side objects of the sm_103a solver.  Included by every .cu file.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/wilson_amg.h"

// ------------------------------------------------------------------ complex
template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};
typedef cx<double> zd;
typedef cx<float> zf;

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cconj(cx<T> a) { return mk(a.re, -a.im); }
// conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// i * a
template <typename T>
__host__ __device__ __forceinline__ cx<T> ci(cx<T> a) { return mk(-a.im, a.re); }
template <typename T>
__host__ __device__ __forceinline__ T cnorm2(cx<T> a) { return a.re * a.re + a.im * a.im; }
// accumulate a * b into acc
template <typename T>
__host__ __device__ __forceinline__ void cfma(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// subtract a * b from acc (the negations fold into the FMAs)
template <typename T>
__host__ __device__ __forceinline__ void cfms(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
// accumulate conj(a) * b into acc
template <typename T>
__host__ __device__ __forceinline__ void cfmac(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

template <typename To, typename From>
__host__ __device__ __forceinline__ cx<To> ccast(cx<From> a) {
  return mk((To)a.re, (To)a.im);
}

// Exact float -> double widening on the integer pipes: for a normal float
// the double has the same sign, the exponent rebiased by 1023 - 127 = 896
// and the 23 mantissa bits shifted up by 29.  Zero, subnormal, inf and NaN
// take the hardware conversion.  (On this GPU the hardware conversion runs
// on the FP64 pipe, which FP64-bound kernels are short of.)
__device__ __forceinline__ double f2d(float f) {
  unsigned u = __float_as_uint(f);
  unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                         ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}
template <typename To, typename From>
struct Widen {
  __device__ __forceinline__ static cx<To> get(cx<From> a) { return ccast<To>(a); }
};
template <>
struct Widen<double, float> {
  __device__ __forceinline__ static cx<double> get(cx<float> a) { return mk(f2d(a.re), f2d(a.im)); }
};
template <typename To, typename From>
__device__ __forceinline__ cx<To> widen(cx<From> a) {
  return Widen<To, From>::get(a);
}

// A complex number held as the unevaluated sum hi + lo of two complex floats
// (|lo| at most half an ulp of hi, per component): about 48 significant bits
// carried on the FP32 pipes.  The storage of the Krylov vectors of the
// Gram-Schmidt process when amg_params.gs_arith = 1.
struct alignas(16) zdf {
  zf hi, lo;
};

// a result computed in cx<T>, stored as Y: itself, widened to zd, or as a
// double-float with lo = 0 (exact in every case)
template <typename Y, typename T>
struct Store;
template <typename T>
struct Store<cx<T>, T> {
  __device__ __forceinline__ static cx<T> get(cx<T> v) { return v; }
};
template <>
struct Store<zd, float> {
  __device__ __forceinline__ static zd get(zf v) { return widen<double>(v); }
};
template <>
struct Store<zdf, float> {
  __device__ __forceinline__ static zdf get(zf v) {
    zdf z;
    z.hi = v;
    z.lo = mk(0.f, 0.f);
    return z;
  }
};
template <typename Y, typename T>
__device__ __forceinline__ Y store_as(cx<T> v) {
  return Store<Y, T>::get(v);
}

// storage of operator coefficients: complex double, complex float or bf16 pair
struct zb {
  __nv_bfloat162 v;
};
template <typename T>
__device__ __forceinline__ cx<T> ld(const zd *p) { return ccast<T>(*p); }
template <typename T>
__device__ __forceinline__ cx<T> ld(const zf *p) { return ccast<T>(*p); }
template <typename T>
__device__ __forceinline__ cx<T> ld(const zb *p) {
  float2 f = __bfloat1622float2(p->v);
  return mk((T)f.x, (T)f.y);
}

// ----------------------------------------------------------------- geometry
// Level l is the even sublattice of an N x N torus (N a power of two).
// site h <-> (x, y): y = h / (N/2), x = 2 (h mod N/2) + (y mod 2).
// Rotated coordinates a = (x+y)/2, b = (x-y)/2; stencil offset
// d = 3 (da+1) + (db+1), (dx, dy) = (da+db, da-db).
#define WL_MAX_DEVICES 64

struct Geo {
  int N, lg;  // N = 1 << lg
  __host__ __device__ __forceinline__ int half() const { return N >> 1; }
  __host__ __device__ __forceinline__ int nsites() const { return (N * N) >> 1; }
  __host__ __device__ __forceinline__ void xy(int h, int &x, int &y) const {
    y = h >> (lg - 1);
    x = ((h & (half() - 1)) << 1) | (y & 1);
  }
  // index of the site (x, y) (any parity-consistent integers; wrapped)
  __host__ __device__ __forceinline__ int idx(int x, int y) const {
    x &= N - 1;
    y &= N - 1;
    return (y << (lg - 1)) | (x >> 1);
  }
  __host__ __device__ __forceinline__ int nb(int x, int y, int d) const {
    int da = d / 3 - 1, db = d % 3 - 1;
    return idx(x + da + db, y + da - db);
  }
};

static inline int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}
static inline Geo make_geo(int N) {
  Geo g;
  g.N = N;
  g.lg = ilog2(N);
  return g;
}

// -------------------------------------------------------------- error state
void wl_set_error(const char *fmt, ...);
// kernel launch accounting (wl_launch_count)
void wl_count_launches(long long n);
extern "C" long long wl_launch_count(void);
#define WL_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t _e = (call);                                                 \
    if (_e != cudaSuccess) {                                                 \
      wl_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                \
                   cudaGetErrorString(_e));                                  \
      return WL_ECUDA;                                                       \
    }                                                                        \
  } while (0)
#define WL_TRY(expr)          \
  do {                        \
    int _rc = (expr);         \
    if (_rc < 0) return _rc;  \
  } while (0)

// ------------------------------------------------------------ device buffer
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  bool own = true;  // false: a view of another object's buffer, never freed or grown here
  int alloc(size_t b);
  void release();
  template <typename T>
  T *as() const { return (T *)p; }
  DBuf view() const {
    DBuf v;
    v.p = p;
    v.bytes = bytes;
    v.own = false;
    return v;
  }
};

// ------------------------------------------------------------ host objects
struct wl_op {
  std::atomic<int> refs{1};  // the caller's handle plus one per live hierarchy
  int N;
  double m, c;
  cudaStream_t stream;  // the library's own non-blocking work stream
  cudaStream_t user;    // the caller's stream given to wilson_create
  int device;           // CUDA device the operator lives on
  cudaEvent_t ev;       // orders the work stream after the caller's stream
  Geo geo;
  DBuf Uf64, Uf32;  // folded links V_mu(z) = sign * U_mu(z) / (2c), [2][N][N]
  uint64_t gauge_hash;
  DBuf scratch;     // small generic scratch for the per-step entry points
};

// one precision copy of a level's operator data
struct LevelOps {
  DBuf A;    // stencil [n][9][2][2]
  DBuf den;  // Kaczmarz denominators ||A e_i||^2, [n][2] (real, T)
  DBuf P;    // interpolation weights to the next level [n][2][4]
};

// launch form of a Kaczmarz sweep on one level, chosen by the autotuner
// (measured) or by the heuristic: form 0 = one launch per colour, 1 = one
// cooperative launch for all colours (param = blocks), 2 = tile-coloured
// kernel (param = right-hand-side chunk R | right-hand sides per thread << 8),
// 3 = block-resident sweeps of a small level (param = right-hand sides per block)
struct KTune {
  int nrhs, prec, form, param;
  float us;  // measured time of one sweep (0 if not measured)
};

struct Level {
  int N, B, n;  // lattice side, cell size to the next level (0 at coarsest), sites
  Geo geo;
  LevelOps op64, op32, opbf;  // FP64 master, FP32 copy, BF16 copy (den in FP32)
  // cycle work vectors, [n][2][nrhs_cap] in the cycle precision
  DBuf x, r, f, t;
  std::vector<KTune> tune;    // autotuned sweep forms per (nrhs, precision)
};

struct wl_amg {
  std::atomic<int> refs{1};  // the caller's handle plus one per server using it
  wl_op *op;
  amg_params prm;
  int L;
  Level lev[8];
  DBuf Ainv;      // coarsest inverse, complex double [nc][nc]
  DBuf Ainv32;    // float copy
  int nc;         // coarsest dimension 2 n_{L-1}
  // Krylov workspace (level-0, [n][2][nrhs_cap])
  int cap;        // right-hand sides the workspace holds
  int cap_prec;   // precision the cycle buffers were sized for
  DBuf V, Z, w, bh, xh, rr;
  DBuf sb, sx;    // device staging of amg_solve_host's b and x (one batch)
  DBuf red;       // reduction partials
  DBuf small;     // per-rhs scalars (Hessenberg, Givens, flags)
  DBuf pinned_small;  // host-pinned mirror of flags
  void *h_small;
  // captured cycle graphs, one per (nrhs, precision)
  struct G {
    int nrhs, prec;
    long long kernels;  // kernel nodes of the graph
    cudaGraphExec_t exec;
  };
  std::vector<G> graphs;
  // second solve lane (amg_params.overlap): a hierarchy that views this one's
  // operators and has its own stream, workspace and graphs; created on demand
  wl_amg *twin = nullptr;
};

// --------------------------------------------------------- internal C++ API
namespace wl {
// lifetime: an operator is freed when its last reference goes (the caller's
// wl_destroy and every hierarchy built on it); a hierarchy likewise (the
// caller's amg_destroy and every server it was added to), so the order in
// which a caller drops its handles does not matter
void op_retain(wl_op *op);
void op_release(wl_op *op);
void amg_retain(wl_amg *a);
void amg_release(wl_amg *a);
int enter(wl_op *op);  // work stream waits for everything queued on the caller's stream
int ensure_workspace(wl_amg *a, int nrhs, int prec);
wl_amg *make_twin(wl_amg *a);  // the second solve lane of a (nullptr on failure, error set)
int level_ops_build_copies(wl_amg *a);
int coarsest_invert(wl_amg *a);
int cycle_run(wl_amg *a, int nrhs, int prec, cudaStream_t s);  // lev[0].f -> lev[0].x
int cycle_prepare(wl_amg *a, int nrhs, int prec, cudaStream_t s, const wl_amg::G **out);  // capture only
int cycle_direct(wl_amg *a, int nrhs, int prec, cudaStream_t s);
int dhat_apply_dev(wl_op *op, const void *x, int x_is_f32, zd *y, int nrhs, cudaStream_t s);
int stencil_apply32_to64(wl_amg *a, const void *x, zd *y, int nrhs, cudaStream_t s);
int stencil_apply32_to_df(wl_amg *a, const void *x, zdf *y, int nrhs, cudaStream_t s);  // lo = 0
int stencil_apply(wl_amg *a, int l, int prec, const void *x, void *y, const void *f, int nrhs,
                  cudaStream_t s);
int kaczmarz_sweeps(wl_amg *a, int l, int prec, void *x, void *r, int nrhs, int sweeps,
                    cudaStream_t s);
int kaczmarz_colour(wl_amg *a, int l, int prec, void *x, void *r, int nrhs, int c, cudaStream_t s);
int kaczmarz_tile(wl_amg *a, int l, int prec, void *x, void *r, int nrhs, int tc, cudaStream_t s, int R = 0);
int autotune_sweeps(wl_amg *a, int nrhs, int prec, cudaStream_t s);  // every level but the coarsest
int tile_timeout_take(cudaStream_t s);  // 1 if a tile launch's bounded wait ran out (flag cleared)
KTune sweep_form_of(wl_amg *a, int l, int prec, int nrhs);
int restrict_op(wl_amg *a, int l, int prec, const void *r, void *fc, int nrhs, cudaStream_t s);
int prolong_op(wl_amg *a, int l, int prec, const void *e, void *x, int nrhs, cudaStream_t s);
int coarsest_apply(wl_amg *a, int prec, const void *f, void *x, int nrhs, cudaStream_t s);
int fgmres_run(wl_amg *a, const zd *bh, zd *xh, int nrhs, double tol, wl_info *info);
int build_dhat_stencil(wl_op *op, zd *A, cudaStream_t s);
int symmetrise_stencil(int N, zd *A, cudaStream_t s);
int compute_den64(int N, const zd *A, double *den, cudaStream_t s);
// layout transposes between the ABI [nrhs][n][2] (FP64) and the internal
// [n][2][nrhs] in precision prec (0 = double, 1 = float)
int to_internal(const zd *src, void *dst, int n2, int nrhs, int prec, cudaStream_t s);
int from_internal(const void *src, zd *dst, int n2, int nrhs, int prec, cudaStream_t s);
size_t prec_bytes(int prec);  // bytes of one complex element of the cycle precision
}  // namespace wl

#define WL_GRID(n, b) ((unsigned)(((n) + (b)-1) / (b)))

// ------------------------------------------- async copies and mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the completion of the mbarrier phase of the given parity, at most
// `ns` nanoseconds (the timer is read once per 32 polls); false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, unsigned long long ns) {
  unsigned long long t0 = gtimer();
  for (;;) {
    for (int i = 0; i < 32; ++i) {
      uint32_t done;
      asm volatile(
          "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
          : "=r"(done)
          : "r"(mb), "r"(parity)
          : "memory");
      if (done) return true;
    }
    if (gtimer() - t0 > ns) return false;
  }
}

__device__ __forceinline__ void mbar_init(uint32_t mb, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mb) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(mb) : "memory");
}
// one arrival that also announces `bytes` of asynchronous copies to come
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mb, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mb),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of
// 16) that completes `bytes` on the mbarrier mb
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mb) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mb)
               : "memory");
}
