// wl_mg.cu -- solve-phase multigrid kernels on the GB300: block-stencil
// apply, multicolour Kaczmarz (Sec. 3.1), Galerkin transfers P^H / P
// (Secs. 3.3, 3.5), the dense coarsest solve (Sec. 4), and the cycle driver
// (Sec. 1 two-grid correction applied recursively).
//
// Vectors use the internal layout [n][2][nrhs] (site, spin, right-hand
// side innermost) so that a warp covers consecutive right-hand sides of one
// site and shares that site's stencil coefficients.
#include <cooperative_groups.h>

#include <algorithm>

#include <atomic>
#include <type_traits>

#include "wl_common.cuh"

namespace cg = cooperative_groups;


// ------------------------------------------------------------ stencil apply
// y = A x, or y = f - A x when f != nullptr (y may alias f); arithmetic in T,
// y stored as Y (the Arnoldi matvec widens an FP32 result to FP64, or keeps
// it as the high part of a double-float).
template <typename T, typename S, typename Y = cx<T>>
__global__ void __launch_bounds__(256) k_stencil(Geo g, const S *__restrict__ A, const cx<T> *__restrict__ x,
                                                 const Y *f, Y *y, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int n = g.nsites();
  if (tid >= (long)n * nrhs) return;
  int h = (int)(tid / nrhs), r = (int)(tid - (long)h * nrhs);
  int px, py;
  g.xy(h, px, py);
  const S *Ah = A + (long)h * 36;
  cx<T> y0 = mk<T>(0, 0), y1 = mk<T>(0, 0);
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    long j = (long)g.nb(px, py, d) * 2 * nrhs + r;
    cx<T> x0 = x[j], x1 = x[j + nrhs];
    cfma(y0, ld<T>(Ah + d * 4 + 0), x0);
    cfma(y0, ld<T>(Ah + d * 4 + 1), x1);
    cfma(y1, ld<T>(Ah + d * 4 + 2), x0);
    cfma(y1, ld<T>(Ah + d * 4 + 3), x1);
  }
  long o = (long)h * 2 * nrhs + r;
  Y z0 = store_as<Y>(y0), z1 = store_as<Y>(y1);
  if constexpr (!std::is_same<Y, zdf>::value) {
    if (f) {
      z0 = f[o] - z0;
      z1 = f[o + nrhs] - z1;
    }
  }
  y[o] = z0;
  y[o + nrhs] = z1;
}

// ---------------------------------------------------------------- Kaczmarz
// One colour of the multicolour sweep.  Colour k = 4 (a mod 4) + (b mod 4);
// item q enumerates a = ka + 4 (q / (N/8)), b = kb + 4 (q mod N/8).
// Column (h, t) of a gamma5-Hermitian A has the entries
//   A_{(j,s),(h,t)} = g_s g_t conj(A[h][d][t][s]),  j = nb(h, d),
// so s = <r, A e> / ||A e||^2 = g_t sum_{d,s} A[h][d][t][s] g_s r_{j,s} / den
// reads only row h of the stencil; then x_(h,t) += omega s and
// r_(j,s) -= omega s g_s g_t conj(A[h][d][t][s]).  Spin 0 precedes spin 1.
__device__ __forceinline__ int kacz_site(const Geo &g, int colour, int q, int &px, int &py) {
  int nb8 = g.N >> 3;
  int a = (colour >> 2) + 4 * (q / nb8);
  int b = (colour & 3) + 4 * (q % nb8);
  px = (a + b) & (g.N - 1);
  py = (a - b) & (g.N - 1);
  return g.idx(px, py);
}

// rv -= g sv conj(a) with g = +1 or -1: the products fold into four FMAs
// (sv conj(a) = (sv.re a.re + sv.im a.im) + i (sv.im a.re - sv.re a.im))
template <typename T>
__device__ __forceinline__ void r_sub(cx<T> &rv, T g, cx<T> sv, cx<T> a) {
  T sr = g * sv.re, si = g * sv.im;  // exact: g = +-1
  rv.re = fma(-sr, a.re, rv.re);
  rv.re = fma(-si, a.im, rv.re);
  rv.im = fma(-si, a.re, rv.im);
  rv.im = fma(sr, a.im, rv.im);
}

// Row inner product of a Kaczmarz step, num = sum_d a_0 r_0 - a_1 r_1
// (complex, a_s = A[h][d][t][s], r_s of neighbour d), as eight independent
// chains: per spin s, P_s = sum_d Re(a_s) (Re r_s, Im r_s) and
// Q_s = sum_d Im(a_s) (Re r_s, Im r_s), then a_s r_s summed is
// (P.re - Q.im, P.im + Q.re).  PAIRED (FP32 only) runs each (re, im) pair of
// chains as one paired FMA (__ffma2_rn), lane for lane the same operation,
// so both forms give the same bits.
template <typename T, bool PAIRED>
__device__ __forceinline__ cx<T> row_dot(const cx<T> (&a)[9][2], const cx<T> (&rv)[9][2]) {
  cx<T> P[2], Q[2];
  if constexpr (PAIRED) {
    static_assert(std::is_same<T, float>::value, "paired FMAs are FP32");
    float2 p2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, q2[2] = {p2[0], p2[0]};
#pragma unroll
    for (int d = 0; d < 9; ++d)
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        float2 v = make_float2(rv[d][sp].re, rv[d][sp].im);
        p2[sp] = __ffma2_rn(make_float2(a[d][sp].re, a[d][sp].re), v, p2[sp]);
        q2[sp] = __ffma2_rn(make_float2(a[d][sp].im, a[d][sp].im), v, q2[sp]);
      }
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      P[sp] = mk(p2[sp].x, p2[sp].y);
      Q[sp] = mk(q2[sp].x, q2[sp].y);
    }
  } else {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) P[sp] = Q[sp] = mk<T>(0, 0);
#pragma unroll
    for (int d = 0; d < 9; ++d)
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        cx<T> v = rv[d][sp], c = a[d][sp];
        P[sp].re = fma(c.re, v.re, P[sp].re);
        P[sp].im = fma(c.re, v.im, P[sp].im);
        Q[sp].re = fma(c.im, v.re, Q[sp].re);
        Q[sp].im = fma(c.im, v.im, Q[sp].im);
      }
  }
  return mk((P[0].re - Q[0].im) - (P[1].re - Q[1].im), (P[0].im + Q[0].re) - (P[1].im + Q[1].re));
}

// one (site, right-hand side) item, one thread
template <typename T, typename S>
__device__ __forceinline__ void kacz_item(const Geo &g, int colour, int q, int rh, const S *__restrict__ A,
                                          const T *__restrict__ den, cx<T> *__restrict__ x,
                                          cx<T> *__restrict__ r, int nrhs, T omega) {
  int px, py;
  int h = kacz_site(g, colour, q, px, py);
  long jj[9];
  cx<T> rv[9][2];
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    jj[d] = (long)g.nb(px, py, d) * 2 * nrhs + rh;
    rv[d][0] = r[jj[d]];
    rv[d][1] = r[jj[d] + nrhs];
  }
  const S *Ah = A + (long)h * 36;
  cx<T> xs[2];
  long xo = (long)h * 2 * nrhs + rh;
  xs[0] = x[xo];
  xs[1] = x[xo + nrhs];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    cx<T> a_[9][2];
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      a_[d][0] = ld<T>(Ah + d * 4 + t * 2 + 0);
      a_[d][1] = ld<T>(Ah + d * 4 + t * 2 + 1);
    }
    // the row inner product as eight independent chains (row_dot), so
    // a thread's step is not one long chain of dependent FMAs
    cx<T> num = row_dot<T, false>(a_, rv);
    T sc = omega / den[2 * h + t];
    if (t) sc = -sc;
    cx<T> sv = sc * num;
    xs[t] = xs[t] + sv;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
#pragma unroll
      for (int s = 0; s < 2; ++s) r_sub(rv[d][s], (s == t) ? (T)1 : (T)-1, sv, a_[d][s]);  // g_s g_t
    }
  }
  x[xo] = xs[0];
  x[xo + nrhs] = xs[1];
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    r[jj[d]] = rv[d][0];
    r[jj[d] + nrhs] = rv[d][1];
  }
}

// one site with a single right-hand side, one warp: lane = 2 d + s holds
// r_(nb(h,d), s); the inner products are warp sums (butterfly, all lanes)
template <typename T, typename S>
__device__ __forceinline__ void kacz_site_warp(const Geo &g, int colour, int q, int lane,
                                               const S *__restrict__ A, const T *__restrict__ den,
                                               cx<T> *__restrict__ x, cx<T> *__restrict__ r, T omega) {
  int px, py;
  int h = kacz_site(g, colour, q, px, py);
  bool act = lane < 18;
  int d = act ? lane >> 1 : 0, s = lane & 1;
  long j = (long)g.nb(px, py, d) * 2 + s;
  cx<T> rv = act ? r[j] : mk<T>(0, 0);
  const S *Ah = A + (long)h * 36 + d * 4;
  T gs = s ? (T)-1 : (T)1;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    cx<T> a_ = act ? ld<T>(Ah + t * 2 + s) : mk<T>(0, 0);
    cx<T> num = mk<T>(0, 0);
    cfma(num, mk<T>(gs * a_.re, gs * a_.im), rv);
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      num.re += __shfl_xor_sync(0xffffffffu, num.re, off);
      num.im += __shfl_xor_sync(0xffffffffu, num.im, off);
    }
    T sc = omega / den[2 * h + t];
    if (t) sc = -sc;
    cx<T> sv = sc * num;
    r_sub(rv, (s == t) ? (T)1 : (T)-1, sv, a_);
    if (lane == 0) {
      long xo = (long)h * 2 + t;
      x[xo] = x[xo] + sv;
    }
  }
  if (act) r[j] = rv;
}

template <typename T, typename S>
__global__ void __launch_bounds__(128) k_kacz(Geo g, int colour, const S *__restrict__ A,
                                              const T *__restrict__ den, cx<T> *__restrict__ x,
                                              cx<T> *__restrict__ r, int nrhs, T omega) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int n16 = g.nsites() >> 4;
  if (tid >= (long)n16 * nrhs) return;
  int q = (int)(tid / nrhs), rh = (int)(tid - (long)q * nrhs);
  kacz_item<T, S>(g, colour, q, rh, A, den, x, r, nrhs, omega);
}

template <typename T, typename S>
__global__ void __launch_bounds__(128) k_kacz_warp(Geo g, int colour, const S *__restrict__ A,
                                                   const T *__restrict__ den, cx<T> *__restrict__ x,
                                                   cx<T> *__restrict__ r, T omega) {
  int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= (g.nsites() >> 4)) return;
  kacz_site_warp<T, S>(g, colour, q, threadIdx.x & 31, A, den, x, r, omega);
}

// asynchronous global -> shared copies (cp.async): the staging loads of a
// block are all in flight at once and waited for together
__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
  else if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// set to 1 by a launch whose bounded wait for its own bulk copies ran out
// (persistent tile form, staged block form)
__device__ int g_tile_timeout;

// Small levels: all colours of `sweeps` sweeps in one launch, a block per
// chunk of RC right-hand sides.  Right-hand sides do not interact, so a block
// owning whole right-hand sides needs only block barriers between colours;
// x and r of its chunk live in shared memory ([n][2][RC] each).  The stencil
// rows and denominators come through the cache, or (STAGE) are staged in
// shared memory as well, so no colour step waits on L2: two 1-D bulk copies
// (the level's whole [n][36] stencil and [n][2] denominators, both contiguous)
// that complete on one mbarrier, with the wait bounded (one second; on a
// timeout g_tile_timeout gets 1 and the block stops without writing).  The
// per-item arithmetic is kacz_item's, so the result equals the other launch
// forms bit for bit.
template <typename T, typename S, bool STAGE>
__global__ void __launch_bounds__(256) k_kacz_block(Geo g, int sweeps, int RC, const S *__restrict__ A,
                                                    const T *__restrict__ den, cx<T> *__restrict__ x,
                                                    cx<T> *__restrict__ r, int nrhs, T omega) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  int n = g.nsites();
  cx<T> *xs = (cx<T> *)sm_raw, *rs = xs + (long)n * 2 * RC;
  S *As = (S *)(rs + (long)n * 2 * RC);  // [n][36] with STAGE
  T *dsm = (T *)(As + (STAGE ? (long)n * 36 : 0));
  uint64_t *mbar = (uint64_t *)(((uintptr_t)(dsm + (STAGE ? 2 * n : 0)) + 7) & ~(uintptr_t)7);
  int r0 = blockIdx.x * RC, rc = min(RC, nrhs - r0);
  int tid = threadIdx.x, nt = blockDim.x;
  if constexpr (STAGE) {
    if (tid == 0) {
      mbar_init(smem_u32(mbar), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
      const uint32_t mb = smem_u32(mbar), ab = (uint32_t)n * 36 * sizeof(S), db = (uint32_t)n * 2 * sizeof(T);
      mbar_arrive_expect_tx(mb, ab + db);
      bulk_g2s(smem_u32(As), A, ab, mb);
      bulk_g2s(smem_u32(dsm), den, db, mb);
    }
  }
  for (int e = tid; e < n * 2 * RC; e += nt) {
    int j = e % RC, row = e / RC;
    bool in = j < rc;
    xs[e] = in ? x[(long)row * nrhs + r0 + j] : mk<T>(0, 0);
    rs[e] = in ? r[(long)row * nrhs + r0 + j] : mk<T>(0, 0);
  }
  if constexpr (STAGE) {
    if (!__syncthreads_and(mbar_wait(smem_u32(mbar), 0, 1000000000ull))) {
      if (tid == 0) atomicExch(&g_tile_timeout, 1);
      return;
    }
  }
  __syncthreads();
  const S *Au = STAGE ? As : A;
  const T *du = STAGE ? dsm : den;
  int n16 = n >> 4;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int c = 0; c < 16; ++c) {
      for (int it = tid; it < n16 * RC; it += nt) {
        int q = it / RC, j = it - q * RC;
        if (j < rc) kacz_item<T, S>(g, c, q, j, Au, du, xs, rs, RC, omega);
      }
      __syncthreads();
    }
  for (int e = tid; e < n * 2 * RC; e += nt) {
    int j = e % RC, row = e / RC;
    if (j < rc) {
      x[(long)row * nrhs + r0 + j] = xs[e];
      r[(long)row * nrhs + r0 + j] = rs[e];
    }
  }
}

// All colours of `sweeps` sweeps in one cooperative launch; a grid-wide
// barrier separates the colours.  wpi = 1: one warp per site (nrhs = 1).
template <typename T, typename S, int WPI>
__global__ void __launch_bounds__(128) k_kacz_coop(Geo g, int sweeps, int wpi, const S *__restrict__ A,
                                                   const T *__restrict__ den, cx<T> *__restrict__ x,
                                                   cx<T> *__restrict__ r, int nrhs, T omega) {
  cg::grid_group grid = cg::this_grid();
  long n16 = g.nsites() >> 4;
  long nthreads = (long)gridDim.x * blockDim.x;
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int c = 0; c < 16; ++c) {
      if (WPI) {
        for (long q = tid >> 5; q < n16; q += nthreads >> 5)
          kacz_site_warp<T, S>(g, c, (int)q, threadIdx.x & 31, A, den, x, r, omega);
      } else {
        for (long it = tid; it < n16 * nrhs; it += nthreads) {
          int q = (int)(it / nrhs), rh = (int)(it - (long)q * nrhs);
          kacz_item<T, S>(g, c, q, rh, A, den, x, r, nrhs, omega);
        }
      }
      grid.sync();
    }
}

// Tile-coloured sweep (reading of Sec. 3.1's parallel ordering, the
// oracle's OR_ORDER_TILE): 8 x 8 tiles in (a, b), tile colour
// (ta mod 2) + 2 (tb mod 2); one launch per tile colour.  A block owns one
// tile and a chunk of right-hand sides: the stencil rows of the tile and r of
// the tile plus its one-site halo are staged in shared memory, the 16 site
// colours run in turn (4 sites each), x of a site is updated in place in
// global memory when its colour comes up (each site is visited once per
// launch), and r is written back.  Same-colour tiles touch disjoint
// (tile + halo) regions, so the write-back does not race.
#define KT 8            // tile side
#define KTH (KT + 2)    // with halo

// two adjacent stored coefficients in one shared-memory load (16 bytes for
// complex float, 8 for a bf16 pair; 2 x 16 for complex double)
template <typename T>
__device__ __forceinline__ void ld2(const zf *p, cx<T> &a0, cx<T> &a1) {
  float4 v = *(const float4 *)p;
  a0 = mk((T)v.x, (T)v.y);
  a1 = mk((T)v.z, (T)v.w);
}
template <typename T>
__device__ __forceinline__ void ld2(const zd *p, cx<T> &a0, cx<T> &a1) {
  double2 u = *(const double2 *)p, v = *(const double2 *)(p + 1);
  a0 = mk((T)u.x, (T)u.y);
  a1 = mk((T)v.x, (T)v.y);
}
template <typename T>
__device__ __forceinline__ void ld2(const zb *p, cx<T> &a0, cx<T> &a1) {
  a0 = ld<T>(p);
  a1 = ld<T>(p + 1);
}

#include "wl_tile_order.h"  // the colour order and window moves of a tile sweep

// origin of tile `t` of tile colour tc
__device__ __forceinline__ void tile_origin(const Geo &g, int tc, int t, int &A0, int &B0) {
  int nb4 = g.N / (4 * KT);  // tiles of one colour along b
  A0 = ((tc & 1) + 2 * (t / nb4)) * KT;
  B0 = ((tc >> 1) + 2 * (t % nb4)) * KT;
}

// stencil rows and denominators of the tile's 64 sites -> shared memory
template <typename T, typename S>
__device__ __forceinline__ void tile_stage_rows(const Geo &g, int A0, int B0, const S *__restrict__ A,
                                                const T *__restrict__ den, S *As, T *ds) {
  const int rowc = 36 * (int)sizeof(S) / 16;  // a row is 36 sizeof(S) bytes, a multiple of 16
  for (int e = threadIdx.x; e < KT * KT * rowc; e += blockDim.x) {
    int ks = e / rowc, c16 = e - ks * rowc;
    int a = A0 + ks / KT, b = B0 + ks % KT;
    long h = g.idx(a + b, a - b);
    cp_async((char *)(As + ks * 36) + 16 * c16, (const char *)(A + h * 36) + 16 * c16, 16);
  }
  for (int e = threadIdx.x; e < KT * KT * 2; e += blockDim.x) {
    int ks = e >> 1;
    int a = A0 + ks / KT, b = B0 + ks % KT;
    long h = g.idx(a + b, a - b);
    cp_async(ds + e, den + 2 * h + (e & 1), (int)sizeof(T));
  }
}

// r_sub as two paired FMAs: (re, im) += (-sr, -si) Re a, then += (-si, sr) Im a
// (the same four roundings in the same order per component)
__device__ __forceinline__ void r_sub_paired(cx<float> &rv, float2 m1, float2 m2, cx<float> a) {
  float2 v = make_float2(rv.re, rv.im);
  v = __ffma2_rn(m1, make_float2(a.re, a.re), v);
  v = __ffma2_rn(m2, make_float2(a.im, a.im), v);
  rv = mk(v.x, v.y);
}

// The 16 colour steps of one tile, in the order tile_step_colour gives
// (thread (k, q): quadrant k, right-hand
// sides r0 + q + j R / RPT), on r of tile + halo staged in rs ([100][2][R],
// visible to every thread after the first barrier below), the step scales
// ds [64][2] and the site-index table hs [100] of the tile; the stencil rows
// run through the ring Ar [3][4][36] (cp.async groups, two steps ahead).
// The caller may have committed cp.async groups of its own before: the wait
// of step 0 completes them too.  Ends with a barrier.
template <typename T, typename S, int R, int RPT, bool PAIRED>
__device__ __forceinline__ void tile_relax(const S *__restrict__ A, cx<T> *__restrict__ x, cx<T> *rs, const T *ds,
                                           S *Ar, const int *hs, int nrhs, int r0, int Rc) {
  constexpr int NT = 4 * R / RPT;
  constexpr int RQ = R / RPT;                     // threads per site
  constexpr int ROWC = 36 * (int)sizeof(S) / 16;  // 16-byte pieces of a stencil row
  const int tid = threadIdx.x;
  // stencil rows of step st (its four sites, quadrant order) -> ring slot st % 3
  auto issue_rows = [&](int st) {
    S *dst = Ar + (st % 3) * 4 * 36;
    const int c = tile_step_colour(st);
    for (int e = tid; e < 4 * ROWC; e += NT) {
      int kk = e / ROWC, c16 = e - kk * ROWC;
      int i = (c >> 2) + 4 * (kk >> 1), j = (c & 3) + 4 * (kk & 1);
      long h = hs[(i + 1) * KTH + j + 1];
      cp_async((char *)(dst + kk * 36) + 16 * c16, (const char *)(A + h * 36) + 16 * c16, 16);
    }
  };
  issue_rows(0);
  cp_async_commit();
  issue_rows(1);
  cp_async_commit();
  const int k = tid / RQ, q0 = tid % RQ;
  bool act[RPT];
#pragma unroll
  for (int m = 0; m < RPT; ++m) act[m] = q0 + m * RQ < Rc;
  // thread (k, q) visits quadrant k of the tile, one site per step; x of the
  // site four steps ahead is loaded while the current step runs (a ring of
  // four), so the HBM latency of x is off the step's critical path
  auto x_at = [&](int st) -> long {
    const int c = tile_step_colour(st);
    int i = (c >> 2) + 4 * (k >> 1), j = (c & 3) + 4 * (k & 1);
    return (long)hs[(i + 1) * KTH + j + 1] * 2 * nrhs + r0 + q0;
  };
  cx<T> xp[4][RPT][2];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    long xo = x_at(u);
#pragma unroll
    for (int m = 0; m < RPT; ++m)
      if (act[m]) {
        xp[u][m][0] = x[xo + m * RQ];
        xp[u][m][1] = x[xo + m * RQ + nrhs];
      }
  }
  // The 3x3 window of r around the site (rows da, columns db) follows the
  // serpentine path: at every step it moves by one row or one column, the
  // six cells that stay are kept in registers, three new ones are read and
  // the three that leave are written back (the whole window after the last
  // step).  No other thread touches a kept cell meanwhile: at every step the
  // four quadrants' windows are disjoint, and the kept cells lie in this
  // thread's windows of both steps.  Two thirds of the shared-memory traffic
  // of r go away; the arithmetic and its order are unchanged.
  cx<T> rv[RPT][9][2];
#pragma unroll
  for (int st = 0; st < 16; ++st) {
    const int c = tile_step_colour(st), u = st & 3;
    cp_async_wait_group<1>();  // everything but the newest group: r, rows of step st
    // One barrier per step: after it every thread has finished step st - 1,
    // so (a) the cells of r written back at the end of step st - 1 are
    // visible, and (b) the ring slot of step st + 2, last read in step st - 1,
    // may be refilled.  Within a step the four quadrants' windows are
    // disjoint, so no thread reads a cell another one writes.
    __syncthreads();
    if (st + 2 < 16) issue_rows(st + 2);
    cp_async_commit();
    int i = (c >> 2) + 4 * (k >> 1), j = (c & 3) + 4 * (k & 1);
    if (act[0]) {
      int ks = i * KT + j;
      const S *Ah = Ar + ((st % 3) * 4 + k) * 36;
      cx<T> ov[RPT][9][2];
#pragma unroll
      for (int m = 0; m < RPT; ++m)
#pragma unroll
        for (int d = 0; d < 9; ++d) {
          ov[m][d][0] = rv[m][d][0];
          ov[m][d][1] = rv[m][d][1];
        }
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        int ls = (i + d / 3) * KTH + (j + d % 3);  // (i + da + 1, j + db + 1)
        const int src = st > 0 ? tile_window_src(st, d) : -1;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
          if (src >= 0) {  // kept from the previous step's window
            rv[m][d][0] = ov[m][src][0];
            rv[m][d][1] = ov[m][src][1];
          } else {
            rv[m][d][0] = rs[(ls * 2) * R + q0 + m * RQ];
            rv[m][d][1] = rs[(ls * 2 + 1) * R + q0 + m * RQ];
          }
        }
      }
      cx<T> sv[RPT][2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        cx<T> a_[9][2];
#pragma unroll
        for (int d = 0; d < 9; ++d) ld2<T>(Ah + d * 4 + t * 2, a_[d][0], a_[d][1]);
        T sc = ds[2 * ks + t];
        if (t) sc = -sc;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
          sv[m][t] = sc * row_dot<T, PAIRED>(a_, rv[m]);
          if constexpr (PAIRED) {
            float sr = sv[m][t].re, si = sv[m][t].im;  // g_s g_t = +1 (s = t), -1 (s != t)
            float2 m1p = make_float2(-sr, -si), m2p = make_float2(-si, sr);
            float2 m1n = make_float2(sr, si), m2n = make_float2(si, -sr);
#pragma unroll
            for (int d = 0; d < 9; ++d)
#pragma unroll
              for (int sp = 0; sp < 2; ++sp)
                r_sub_paired(rv[m][d][sp], sp == t ? m1p : m1n, sp == t ? m2p : m2n, a_[d][sp]);
          } else {
#pragma unroll
            for (int d = 0; d < 9; ++d)
#pragma unroll
              for (int sp = 0; sp < 2; ++sp) r_sub(rv[m][d][sp], (sp == t) ? (T)1 : (T)-1, sv[m][t], a_[d][sp]);
          }
        }
      }
      long xo = x_at(st), xn = st + 4 < 16 ? x_at(st + 4) : 0;
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        if (!act[m]) continue;
        x[xo + m * RQ] = xp[u][m][0] + sv[m][0];
        x[xo + m * RQ + nrhs] = xp[u][m][1] + sv[m][1];
        if (st + 4 < 16) {
          xp[u][m][0] = x[xn + m * RQ];
          xp[u][m][1] = x[xn + m * RQ + nrhs];
        }
      }
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        if (!tile_window_leaves(st, d)) continue;  // kept for the next step
        int ls = (i + d / 3) * KTH + (j + d % 3);
#pragma unroll
        for (int m = 0; m < RPT; ++m)
          if (act[m]) {
            rs[(ls * 2) * R + q0 + m * RQ] = rv[m][d][0];
            rs[(ls * 2 + 1) * R + q0 + m * RQ] = rv[m][d][1];
          }
      }
    }
  }
  __syncthreads();
}

// The colour steps of tile_relax with each (site, right-hand side) item split
// over a pair of adjacent lanes (FP32, paired FMAs): lane p of the pair holds
// spin component p of r at the site's nine neighbours, forms that spin's
// partial row products P_p, Q_p (the chains row_dot forms per spin, in the
// same order), takes the partner's by one shuffle, and both lanes combine
// them in row_dot's order, so every value matches tile_relax bit for bit.
// Lane p then updates its component of r and x component p.  Half the
// instructions per thread and twice the warps per tile: for levels where a
// launch has few tiles and each step's latency, not issue, sets the time.
// Thread (k, q, p) = (tid / 2R, (tid % 2R) / 2, tid % 2).  Every lane runs
// the arithmetic (lanes past the chunk on stale shared memory, results
// discarded) so that the shuffles see full warps.  Ends with a barrier.
template <typename S, int R>
__device__ __forceinline__ void tile_relax_split(const S *__restrict__ A, zf *__restrict__ x, zf *rs,
                                                 const float *ds, S *Ar, const int *hs, int nrhs, int r0,
                                                 int Rc) {
  constexpr int NT = 8 * R;
  constexpr int ROWC = 36 * (int)sizeof(S) / 16;
  const int tid = threadIdx.x;
  auto issue_rows = [&](int st) {
    S *dst = Ar + (st % 3) * 4 * 36;
    const int c = tile_step_colour(st);
    for (int e = tid; e < 4 * ROWC; e += NT) {
      int kk = e / ROWC, c16 = e - kk * ROWC;
      int i = (c >> 2) + 4 * (kk >> 1), j = (c & 3) + 4 * (kk & 1);
      long h = hs[(i + 1) * KTH + j + 1];
      cp_async((char *)(dst + kk * 36) + 16 * c16, (const char *)(A + h * 36) + 16 * c16, 16);
    }
  };
  issue_rows(0);
  cp_async_commit();
  issue_rows(1);
  cp_async_commit();
  const int k = tid / (2 * R), q0 = (tid % (2 * R)) >> 1, p = tid & 1;
  const bool act = q0 < Rc;
  auto x_at = [&](int st) -> long {
    const int c = tile_step_colour(st);
    int i = (c >> 2) + 4 * (k >> 1), j = (c & 3) + 4 * (k & 1);
    return (long)hs[(i + 1) * KTH + j + 1] * 2 * nrhs + (long)p * nrhs + r0 + q0;
  };
  zf xp[4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (act) xp[u] = x[x_at(u)];
  zf rv[9];
#pragma unroll
  for (int st = 0; st < 16; ++st) {
    {
      const int c = tile_step_colour(st), u = st & 3;
      cp_async_wait_group<1>();
      __syncthreads();  // one barrier per step, as in tile_relax
      if (st + 2 < 16) issue_rows(st + 2);
      cp_async_commit();
      int i = (c >> 2) + 4 * (k >> 1), j = (c & 3) + 4 * (k & 1);
      int ks = i * KT + j;
      const S *Ah = Ar + ((st % 3) * 4 + k) * 36;
      zf ov[9];
#pragma unroll
      for (int d = 0; d < 9; ++d) ov[d] = rv[d];
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        int ls = (i + d / 3) * KTH + (j + d % 3);
        const int src = st > 0 ? tile_window_src(st, d) : -1;
        if (src >= 0) rv[d] = ov[src];
        else rv[d] = rs[(ls * 2 + p) * R + q0];
      }
      zf sv[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        zf a_[9];
#pragma unroll
        for (int d = 0; d < 9; ++d) a_[d] = ld<float>(Ah + d * 4 + t * 2 + p);
        float sc = ds[2 * ks + t];
        if (t) sc = -sc;
        // this lane's spin: the chains of row_dot for sp = p
        float2 pp = make_float2(0.f, 0.f), qq = pp;
#pragma unroll
        for (int d = 0; d < 9; ++d) {
          float2 v = make_float2(rv[d].re, rv[d].im);
          pp = __ffma2_rn(make_float2(a_[d].re, a_[d].re), v, pp);
          qq = __ffma2_rn(make_float2(a_[d].im, a_[d].im), v, qq);
        }
        float2 po = make_float2(__shfl_xor_sync(0xffffffffu, pp.x, 1), __shfl_xor_sync(0xffffffffu, pp.y, 1));
        float2 qo = make_float2(__shfl_xor_sync(0xffffffffu, qq.x, 1), __shfl_xor_sync(0xffffffffu, qq.y, 1));
        float2 P0 = p ? po : pp, Q0 = p ? qo : qq, P1 = p ? pp : po, Q1 = p ? qq : qo;
        zf num = mk((P0.x - Q0.y) - (P1.x - Q1.y), (P0.y + Q0.x) - (P1.y + Q1.x));
        sv[t] = sc * num;
        float sr = sv[t].re, si = sv[t].im;  // g_s g_t = +1 (s = t), -1 (s != t)
        float2 m1 = p == t ? make_float2(-sr, -si) : make_float2(sr, si);
        float2 m2 = p == t ? make_float2(-si, sr) : make_float2(si, -sr);
#pragma unroll
        for (int d = 0; d < 9; ++d) r_sub_paired(rv[d], m1, m2, a_[d]);
      }
      if (act) {
        long xo = x_at(st);
        x[xo] = xp[u] + (p ? sv[1] : sv[0]);
        if (st + 4 < 16) xp[u] = x[x_at(st + 4)];
      }
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        if (!tile_window_leaves(st, d)) continue;  // kept for the next step
        int ls = (i + d / 3) * KTH + (j + d % 3);
        rs[(ls * 2 + p) * R + q0] = rv[d];
      }
    }
  }
  __syncthreads();
}

// Several right-hand sides: a block of 4 R / RPT threads, thread (k, q) owns
// site k of the current colour step and right-hand sides r0 + q + j R / RPT
// (j < RPT), which share the stencil coefficients and the index arithmetic.
// Shared memory: r of tile + halo [100][2][R], omega / den [64][2], a ring
// of three colour steps' stencil rows [3][4][36] filled by cp.async two
// steps ahead, and the site indices of tile + halo [100] (about 55 KB at
// R = 32, so four blocks fit an SM).  vec: r rows
// start on 16-byte boundaries (16-byte copies), else one complex per copy.
// Every right-hand side sees the same operations in the same order for any
// R, RPT and PAIRED (paired FP32 FMAs in row_dot and r_sub_paired), so the
// variants agree bit for bit.
// SPLIT: each item over a pair of lanes (tile_relax_split), 8 R threads.
// Launch bounds: one right-hand side per thread keeps 128 registers (512
// threads per SM, four blocks of 128 at R = 32, as shared memory allows);
// the split form keeps 85 (768 threads per SM).
template <typename T, typename S, int R, int RPT, bool PAIRED, bool SPLIT = false>
__global__ void __launch_bounds__(SPLIT ? 8 * R : 4 * R / RPT, SPLIT ? 768 / (8 * R) : (RPT == 1 ? R / 8 : 1))
    k_kacz_tile(Geo g, int tc, const S *__restrict__ A, const T *__restrict__ den, cx<T> *__restrict__ x,
                cx<T> *__restrict__ r, int nrhs, int vec, T omega) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cx<T> *rs = (cx<T> *)sm_raw;
  T *ds = (T *)(rs + KTH * KTH * 2 * R);
  S *Ar = (S *)(ds + KT * KT * 2);
  int *hs = (int *)(Ar + 3 * 4 * 36);  // site index of tile + halo site ls = KTH (i + 1) + (j + 1)
  constexpr int NT = SPLIT ? 8 * R : 4 * R / RPT;
  constexpr int E = 16 / (int)sizeof(cx<T>);  // complex numbers per 16-byte copy
  constexpr int CPR = R / E;                   // 16-byte pieces per staged row
  int A0, B0;
  tile_origin(g, tc, blockIdx.x, A0, B0);
  int r0 = blockIdx.y * R;
  int Rc = min(R, nrhs - r0);
  int tid = threadIdx.x;
  for (int ls = tid; ls < KTH * KTH; ls += NT) {
    int a = A0 + ls / KTH - 1, b = B0 + ls % KTH - 1;
    hs[ls] = g.idx(a + b, a - b);
  }
  __syncthreads();
  // group 0: r of tile + halo
  if (vec) {
    for (int e = tid; e < KTH * KTH * 2 * CPR; e += NT) {
      int c = e % CPR, row = e / CPR;
      if (c * E >= Rc) continue;
      long h = hs[row >> 1];
      cp_async(rs + row * R + c * E, r + (h * 2 + (row & 1)) * nrhs + r0 + c * E, 16);
    }
  } else {
    for (int e = tid; e < KTH * KTH * 2 * R; e += NT) {
      int q = e % R, row = e / R;
      if (q >= Rc) continue;
      long h = hs[row >> 1];
      cp_async(rs + e, r + (h * 2 + (row & 1)) * nrhs + r0 + q, (int)sizeof(cx<T>));
    }
  }
  for (int e = tid; e < KT * KT * 2; e += NT) {
    int ks = e >> 1;
    long h = hs[(ks / KT + 1) * KTH + ks % KT + 1];
    ds[e] = omega / den[2 * h + (e & 1)];  // the step scale, once per site and spin
  }
  cp_async_commit();
  if constexpr (SPLIT) {
    static_assert(std::is_same<T, float>::value && PAIRED && RPT == 1, "the split form is FP32 with paired FMAs");
    tile_relax_split<S, R>(A, x, rs, ds, Ar, hs, nrhs, r0, Rc);
  } else {
    tile_relax<T, S, R, RPT, PAIRED>(A, x, rs, ds, Ar, hs, nrhs, r0, Rc);
  }
  // write r back (tile and halo)
  if (vec) {
    for (int e = tid; e < KTH * KTH * 2 * CPR; e += NT) {
      int c = e % CPR, row = e / CPR;
      if (c * E >= Rc) continue;
      long h = hs[row >> 1];
      *(int4 *)(r + (h * 2 + (row & 1)) * nrhs + r0 + c * E) = *(const int4 *)(rs + row * R + c * E);
    }
  } else {
    for (int e = tid; e < KTH * KTH * 2 * R; e += NT) {
      int q2 = e % R, row = e / R;
      if (q2 >= Rc) continue;
      long h = hs[row >> 1];
      r[(h * 2 + (row & 1)) * nrhs + r0 + q2] = rs[e];
    }
  }
}

// Persistent form of k_kacz_tile (launch parameter bit 0x1000): a block per
// SM slot takes the items (tile, chunk of R right-hand sides) w = blockIdx.x
// + i gridDim.x of the launch in turn, with r of tile + halo double-buffered:
// while a tile relaxes, one warp has the next item's r on its way as 1-D bulk
// copies (one per site and spin, R complex numbers each) that complete on
// that buffer's mbarrier, so DRAM reads overlap the colour steps instead of
// preceding them.  The colour steps are tile_relax, the same operations in
// the same order as the one-tile-per-block form.  Needs full chunks whose
// rows start on 16-byte boundaries (vec and nrhs a multiple of R; the
// launcher checks).  Tiles of one colour have disjoint tile + halo regions,
// so prefetching one while another is written back cannot race.  The wait
// for a buffer is bounded (one second); on a timeout g_tile_timeout gets 1
// and the block stops.

template <typename T, typename S, int R, int RPT, bool PAIRED>
__global__ void __launch_bounds__(4 * R / RPT) k_kacz_tile_p(Geo g, int tc, const S *__restrict__ A,
                                                             const T *__restrict__ den, cx<T> *__restrict__ x,
                                                             cx<T> *__restrict__ r, int nrhs, T omega, int ntiles) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cx<T> *rs = (cx<T> *)sm_raw;  // [2][100][2][R]
  T *ds = (T *)(rs + 2 * KTH * KTH * 2 * R);
  S *Ar = (S *)(ds + KT * KT * 2);
  int *hs = (int *)(Ar + 3 * 4 * 36);
  uint64_t *mbar = (uint64_t *)(((uintptr_t)(hs + KTH * KTH) + 7) & ~(uintptr_t)7);
  constexpr int NT = 4 * R / RPT;
  constexpr uint32_t ROWB = R * sizeof(cx<T>);  // bytes of one staged row (site, spin)
  const int tid = threadIdx.x;
  const int nitems = ntiles * (nrhs / R);
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // warp 0: the bulk copies of item w's r into buffer b
  auto fetch = [&](int w, int b) {
    if (tid >= 32) return;
    int A0, B0;
    tile_origin(g, tc, w % ntiles, A0, B0);
    const int rr0 = (w / ntiles) * R;
    const uint32_t mb = smem_u32(&mbar[b]);
    if (tid == 0) mbar_arrive_expect_tx(mb, (uint32_t)(KTH * KTH * 2) * ROWB);
    __syncwarp();
    cx<T> *dst = rs + (size_t)b * KTH * KTH * 2 * R;
    for (int row = tid; row < KTH * KTH * 2; row += 32) {
      int ls = row >> 1, a = A0 + ls / KTH - 1, bb = B0 + ls % KTH - 1;
      long h = g.idx(a + bb, a - bb);
      bulk_g2s(smem_u32(dst + row * R), r + (h * 2 + (row & 1)) * nrhs + rr0, ROWB, mb);
    }
  };
  if ((int)blockIdx.x < nitems) fetch(blockIdx.x, 0);
  int i = 0;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x, ++i) {
    const int b = i & 1;
    int A0, B0;
    tile_origin(g, tc, w % ntiles, A0, B0);
    const int r0 = (w / ntiles) * R;
    for (int ls = tid; ls < KTH * KTH; ls += NT) {
      int a = A0 + ls / KTH - 1, bb = B0 + ls % KTH - 1;
      hs[ls] = g.idx(a + bb, a - bb);
    }
    for (int e = tid; e < KT * KT * 2; e += NT) {
      int ks = e >> 1, a = A0 + ks / KT, bb = B0 + ks % KT;
      ds[e] = omega / den[2 * (long)g.idx(a + bb, a - bb) + (e & 1)];
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait(smem_u32(&mbar[b]), (uint32_t)((i >> 1) & 1), 1000000000ull))) {
      if (tid == 0) atomicExch(&g_tile_timeout, 1);
      break;
    }
    if (w + (int)gridDim.x < nitems) fetch(w + gridDim.x, b ^ 1);  // that buffer was freed after item i - 1
    cx<T> *rb = rs + (size_t)b * KTH * KTH * 2 * R;
    tile_relax<T, S, R, RPT, PAIRED>(A, x, rb, ds, Ar, hs, nrhs, r0, R);
    // write r back (tile and halo), 16 bytes per store
    constexpr int E = 16 / (int)sizeof(cx<T>), CPR = R / E;
    for (int e = tid; e < KTH * KTH * 2 * CPR; e += NT) {
      int c = e % CPR, row = e / CPR;
      long h = hs[row >> 1];
      *(int4 *)(r + (h * 2 + (row & 1)) * nrhs + r0 + c * E) = *(const int4 *)(rb + row * R + c * E);
    }
    // the next bulk copy into this buffer (item i + 2) is an async-proxy write after these reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
}

// One right-hand side: a warp per site of the colour step, lane = 2 d + s
// holds one term of the row's inner product; shared memory: A rows, den and
// r of tile + halo [100][2].
template <typename T, typename S>
__global__ void __launch_bounds__(128) k_kacz_tile1(Geo g, int tc, const S *__restrict__ A,
                                                    const T *__restrict__ den, cx<T> *__restrict__ x,
                                                    cx<T> *__restrict__ r, T omega) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  S *As = (S *)sm_raw;
  T *ds = (T *)(As + KT * KT * 36);
  cx<T> *rs = (cx<T> *)(ds + KT * KT * 2);
  int A0, B0;
  tile_origin(g, tc, blockIdx.x, A0, B0);
  int tid = threadIdx.x;
  tile_stage_rows<T, S>(g, A0, B0, A, den, As, ds);
  for (int e = tid; e < KTH * KTH * 2; e += blockDim.x) {
    int ls = e >> 1;
    int a = A0 + ls / KTH - 1, b = B0 + ls % KTH - 1;
    long h = g.idx(a + b, a - b);
    cp_async(rs + e, r + h * 2 + (e & 1), (int)sizeof(cx<T>));
  }
  cp_async_wait_all();
  __syncthreads();
  const int k = tid >> 5, lane = tid & 31;
  // lane 0 of warp k holds x of its quadrant's sites four steps ahead
  auto x_at = [&](int st) -> long {
    const int c = tile_step_colour(st);
    int i = (c >> 2) + 4 * (k >> 1), j = (c & 3) + 4 * (k & 1);
    return (long)g.idx(A0 + i + B0 + j, A0 + i - B0 - j) * 2;
  };
  cx<T> xp[4][2];
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (k < 4 && lane == 0) {
      xp[u][0] = x[x_at(u)];
      xp[u][1] = x[x_at(u) + 1];
    }
  for (int c0 = 0; c0 < 16; c0 += 4) {
#pragma unroll
   for (int u = 0; u < 4; ++u) {
    const int st = c0 + u, c = tile_step_colour(st);
    if (k < 4) {
      int i = (c >> 2) + 4 * (k >> 1), j = (c & 3) + 4 * (k & 1);
      int ks = i * KT + j;
      bool act = lane < 18;
      int d = act ? lane >> 1 : 0, sp = lane & 1;
      int ls = (i + d / 3) * KTH + (j + d % 3);  // (i + da + 1, j + db + 1)
      cx<T> rv = act ? rs[ls * 2 + sp] : mk<T>(0, 0);
      const S *Ah = As + ks * 36 + d * 4;
      T gs = sp ? (T)-1 : (T)1;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        cx<T> a_ = act ? ld<T>(Ah + t * 2 + sp) : mk<T>(0, 0);
        cx<T> num = mk<T>(0, 0);
        cfma(num, mk<T>(gs * a_.re, gs * a_.im), rv);
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          num.re += __shfl_xor_sync(0xffffffffu, num.re, off);
          num.im += __shfl_xor_sync(0xffffffffu, num.im, off);
        }
        T sc = omega / ds[2 * ks + t];
        if (t) sc = -sc;
        cx<T> sv = sc * num;
        r_sub(rv, (sp == t) ? (T)1 : (T)-1, sv, a_);
        if (lane == 0) x[x_at(st) + t] = xp[u][t] + sv;
      }
      if (lane == 0 && st + 4 < 16) {
        xp[u][0] = x[x_at(st + 4)];
        xp[u][1] = x[x_at(st + 4) + 1];
      }
      if (act) rs[ls * 2 + sp] = rv;
    }
    __syncthreads();
   }
  }
  for (int e = tid; e < KTH * KTH * 2; e += blockDim.x) {
    int ls = e >> 1;
    int a = A0 + ls / KTH - 1, b = B0 + ls % KTH - 1;
    long h = g.idx(a + b, a - b);
    r[h * 2 + (e & 1)] = rs[e];
  }
}

// ---------------------------------------------------------------- transfers
// fc = P^H r: coarse site hc gathers the fine points of the (2B-1)^2 box
// around its C point; a fine point at offset (da, db) sees hc as its cell
// corner k = [da < 0] + 2 [db < 0].
template <typename T, typename S>
__global__ void k_restrict(Geo gf, Geo gc, int lgB, const S *__restrict__ P,
                           const cx<T> *__restrict__ r, cx<T> *__restrict__ fc, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int nc = gc.nsites();
  if (tid >= (long)nc * nrhs) return;
  int hc = (int)(tid / nrhs), rh = (int)(tid - (long)hc * nrhs);
  int xc, yc;
  gc.xy(hc, xc, yc);
  int B = 1 << lgB;
  int X = xc << lgB, Y = yc << lgB;
  cx<T> a0 = mk<T>(0, 0), a1 = mk<T>(0, 0);
  for (int da = -(B - 1); da <= B - 1; ++da)
    for (int db = -(B - 1); db <= B - 1; ++db) {
      int hf = gf.idx(X + da + db, Y + da - db);
      int k = (da < 0 ? 1 : 0) + (db < 0 ? 2 : 0);
      long j = (long)hf * 2 * nrhs + rh;
      cfmac(a0, ld<T>(P + (long)hf * 8 + k), r[j]);
      cfmac(a1, ld<T>(P + (long)hf * 8 + 4 + k), r[j + nrhs]);
    }
  long o = (long)hc * 2 * nrhs + rh;
  fc[o] = a0;
  fc[o + nrhs] = a1;
}

// x += P e: fine site (a, b) with cell origin (a0, b0) = B floor((a, b)/B)
// interpolates from the existing corners (a0 + ka B, b0 + kb B).
template <typename T, typename S>
__global__ void k_prolong(Geo gf, Geo gc, int lgB, const S *__restrict__ P,
                          const cx<T> *__restrict__ e, cx<T> *__restrict__ x, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int nf = gf.nsites();
  if (tid >= (long)nf * nrhs) return;
  int hf = (int)(tid / nrhs), rh = (int)(tid - (long)hf * nrhs);
  int px, py;
  gf.xy(hf, px, py);
  int B = 1 << lgB;
  int a = (px + py) >> 1, b = (px - py) >> 1;
  int a0 = a & ~(B - 1), b0 = b & ~(B - 1);
  int ra = a - a0, rb = b - b0;
  long o = (long)hf * 2 * nrhs + rh;
  cx<T> x0 = x[o], x1 = x[o + nrhs];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int ka = k & 1, kb = k >> 1;
    if ((ka && !ra) || (kb && !rb)) continue;
    int ac = a0 + ka * B, bc = b0 + kb * B;
    int xf = (ac + bc) & (gf.N - 1), yf = (ac - bc) & (gf.N - 1);
    long j = (long)gc.idx(xf >> lgB, yf >> lgB) * 2 * nrhs + rh;
    cfma(x0, ld<T>(P + (long)hf * 8 + k), e[j]);
    cfma(x1, ld<T>(P + (long)hf * 8 + 4 + k), e[j + nrhs]);
  }
  x[o] = x0;
  x[o + nrhs] = x1;
}

// x = Ainv f on the coarsest level, FP64 arithmetic: 8 rows per block, one
// warp per row, lanes stride the columns, shuffle reduction.
template <typename T>
__global__ void __launch_bounds__(256) k_coarsest(int nc, const zd *__restrict__ Ainv,
                                                  const cx<T> *__restrict__ f, cx<T> *__restrict__ x,
                                                  int nrhs) {
  int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  int rh = blockIdx.y;
  if (row >= nc) return;
  zd acc = mk(0.0, 0.0);
  const zd *Ar = Ainv + (long)row * nc;
  for (int j = lane; j < nc; j += 32) cfma(acc, Ar[j], ccast<double>(f[(long)j * nrhs + rh]));
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    acc.re += __shfl_down_sync(0xffffffffu, acc.re, off);
    acc.im += __shfl_down_sync(0xffffffffu, acc.im, off);
  }
  if (lane == 0) x[(long)row * nrhs + rh] = ccast<T>(acc);
}

template <typename T>
__global__ void k_axpy_inplace(cx<T> *__restrict__ y, const cx<T> *__restrict__ x, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = y[i] + x[i];
}

namespace wl {

static const LevelOps &ops_of(const Level &L, int prec) {
  return prec == WL_FP64 ? L.op64 : prec == WL_FP32 ? L.op32 : L.opbf;
}

int kaczmarz_colour(wl_amg *a, int l, int prec, void *x, void *r, int nrhs, int c, cudaStream_t s) {
  const Level &L = a->lev[l];
  const LevelOps &o = ops_of(L, prec);
  long n16 = L.n >> 4;
  wl_count_launches(1);
  if (nrhs == 1) {
    unsigned grid = WL_GRID(n16 * 32, 128);
    if (prec == WL_FP64)
      k_kacz_warp<double, zd><<<grid, 128, 0, s>>>(L.geo, c, o.A.as<zd>(), o.den.as<double>(), (zd *)x, (zd *)r, a->prm.omega);
    else if (prec == WL_FP32)
      k_kacz_warp<float, zf><<<grid, 128, 0, s>>>(L.geo, c, o.A.as<zf>(), o.den.as<float>(), (zf *)x, (zf *)r, (float)a->prm.omega);
    else
      k_kacz_warp<float, zb><<<grid, 128, 0, s>>>(L.geo, c, o.A.as<zb>(), o.den.as<float>(), (zf *)x, (zf *)r, (float)a->prm.omega);
    return WL_OK;
  }
  unsigned grid = WL_GRID(n16 * nrhs, 128);
  if (prec == WL_FP64)
    k_kacz<double, zd><<<grid, 128, 0, s>>>(L.geo, c, o.A.as<zd>(), o.den.as<double>(), (zd *)x, (zd *)r, nrhs, a->prm.omega);
  else if (prec == WL_FP32)
    k_kacz<float, zf><<<grid, 128, 0, s>>>(L.geo, c, o.A.as<zf>(), o.den.as<float>(), (zf *)x, (zf *)r, nrhs, (float)a->prm.omega);
  else
    k_kacz<float, zb><<<grid, 128, 0, s>>>(L.geo, c, o.A.as<zb>(), o.den.as<float>(), (zf *)x, (zf *)r, nrhs, (float)a->prm.omega);
  return WL_OK;
}

// resident blocks of 128 threads for the cooperative sweep (cached per
// kernel instance and device)
template <typename T, typename S>
static int coop_blocks() {
  static std::atomic<int> cached[WL_MAX_DEVICES];  // per device, 0 = not yet known
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= WL_MAX_DEVICES) return 0;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    int sms = 0, p0 = 0, p1 = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p0, k_kacz_coop<T, S, 0>, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_kacz_coop<T, S, 1>, 128, 0);
    v = sms * std::min(p0, p1);
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// raise a kernel's dynamic shared-memory limit once per device
static int set_smem_limit(const void *fn, size_t bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  WL_CUDA(cudaGetDevice(&dev));
  unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_acquire) & bit)) {
    WL_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.fetch_or(bit, std::memory_order_acq_rel);
  }
  return WL_OK;
}

template <typename T, typename S>
static int launch_coop(const Level &L, const LevelOps &o, int sweeps, void *x, void *r, int nrhs, double omega,
                       cudaStream_t s, int want_blocks) {
  long n16 = L.n >> 4;
  int wpi = nrhs == 1;
  long threads = wpi ? n16 * 32 : n16 * nrhs;
  int maxb = coop_blocks<T, S>();  // all blocks must be resident at once
  int blocks = (int)std::min<long>(WL_GRID(threads, 128), (long)maxb);
  if (want_blocks > 0) blocks = std::min(blocks, want_blocks);
  if (blocks < 1) return WL_EINVAL;
  Geo g = L.geo;
  const S *A = o.A.as<S>();
  const T *den = o.den.as<T>();
  cx<T> *xx = (cx<T> *)x, *rr = (cx<T> *)r;
  T om = (T)omega;
  void *args[] = {&g, &sweeps, &wpi, (void *)&A, (void *)&den, &xx, &rr, &nrhs, &om};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(128);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const void *fn = wpi ? (const void *)k_kacz_coop<T, S, 1> : (const void *)k_kacz_coop<T, S, 0>;
  WL_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
  return WL_OK;
}

// Fine-grid stencil apply with shared-memory tiles: a block owns an 8 x 8
// tile in (a, b) and a chunk of R right-hand sides; x of tile + halo and the
// tile's stencil rows are staged once (cp.async), so each x value crosses
// L2 once per tile instead of once per neighbour.  Same arithmetic, in the
// same order, as k_stencil.  x must not alias y.
template <typename T, typename S, typename Y, int R, int WF>
__global__ void __launch_bounds__(256) k_stencil_tile(Geo g, const S *__restrict__ A, const cx<T> *__restrict__ x,
                                                      const Y *f, Y *y, int nrhs, int vec) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cx<T> *xs = (cx<T> *)sm_raw;                  // [100][2][R]
  S *As = (S *)(xs + KTH * KTH * 2 * R);        // [64][36]
  int *hs = (int *)(As + KT * KT * 36);         // [100] site indices of tile + halo
  constexpr int NT = 256;
  constexpr int E = 16 / (int)sizeof(cx<T>);
  constexpr int CPR = R / E;
  constexpr int ROWC = 36 * (int)sizeof(S) / 16;
  int nbt = g.N / (2 * KT);  // tiles along b
  int A0 = (blockIdx.x / nbt) * KT, B0 = (blockIdx.x % nbt) * KT;
  int r0 = blockIdx.y * R, Rc = min(R, nrhs - r0);
  int tid = threadIdx.x;
  for (int ls = tid; ls < KTH * KTH; ls += NT) {
    int a = A0 + ls / KTH - 1, b = B0 + ls % KTH - 1;
    hs[ls] = g.idx(a + b, a - b);
  }
  __syncthreads();
  if (vec) {
    for (int e = tid; e < KTH * KTH * 2 * CPR; e += NT) {
      int c = e % CPR, row = e / CPR;
      if (c * E >= Rc) continue;
      long h = hs[row >> 1];
      cp_async(xs + row * R + c * E, x + (h * 2 + (row & 1)) * nrhs + r0 + c * E, 16);
    }
  } else {
    for (int e = tid; e < KTH * KTH * 2 * R; e += NT) {
      int q = e % R, row = e / R;
      if (q >= Rc) continue;
      long h = hs[row >> 1];
      cp_async(xs + e, x + (h * 2 + (row & 1)) * nrhs + r0 + q, (int)sizeof(cx<T>));
    }
  }
  for (int e = tid; e < KT * KT * ROWC; e += NT) {
    int ks = e / ROWC, c16 = e - ks * ROWC;
    long h = hs[(ks / KT + 1) * KTH + ks % KT + 1];
    cp_async((char *)(As + ks * 36) + 16 * c16, (const char *)(A + h * 36) + 16 * c16, 16);
  }
  // f of this thread's outputs is loaded while the staging copies fly
  constexpr int PER = KT * KT * R / NT;  // outputs per thread
  Y fv[WF ? PER : 1][2];
  if constexpr (WF) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      int it = tid + u * NT, q = it % R, ks = it / R;
      if (q < Rc) {
        long o = (long)hs[(ks / KT + 1) * KTH + ks % KT + 1] * 2 * nrhs + r0 + q;
        fv[u][0] = f[o];
        fv[u][1] = f[o + nrhs];
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    int it = tid + u * NT;
    int q = it % R, ks = it / R;
    if (q >= Rc) continue;
    int i = ks / KT, j = ks % KT;
    const S *Ah = As + ks * 36;
    cx<T> y0 = mk<T>(0, 0), y1 = mk<T>(0, 0);
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      int ls = (i + d / 3) * KTH + (j + d % 3);  // (i + da + 1, j + db + 1)
      cx<T> x0 = xs[(ls * 2) * R + q], x1 = xs[(ls * 2 + 1) * R + q];
      cfma(y0, ld<T>(Ah + d * 4 + 0), x0);
      cfma(y0, ld<T>(Ah + d * 4 + 1), x1);
      cfma(y1, ld<T>(Ah + d * 4 + 2), x0);
      cfma(y1, ld<T>(Ah + d * 4 + 3), x1);
    }
    long o = (long)hs[(i + 1) * KTH + j + 1] * 2 * nrhs + r0 + q;
    Y z0 = store_as<Y>(y0), z1 = store_as<Y>(y1);
    if constexpr (WF) {
      z0 = fv[u][0] - z0;
      z1 = fv[u][1] - z1;
    }
    y[o] = z0;
    y[o + nrhs] = z1;
  }
}

template <typename T, typename S>
static size_t stencil_tile_smem(int R) {
  return (size_t)KTH * KTH * 2 * R * sizeof(cx<T>) + (size_t)KT * KT * 36 * sizeof(S) + KTH * KTH * sizeof(int);
}

template <typename T, typename S, typename Y, int R>
static int launch_stencil_tile_r(const Level &L, const S *A, const void *x, const void *f, void *y, int nrhs,
                                 cudaStream_t s) {
  size_t smem = stencil_tile_smem<T, S>(R);
  static std::atomic<unsigned long long> limit_set[2];
  int vec = ((uintptr_t)x % 16 == 0) && (sizeof(T) == 8 || nrhs % 2 == 0);
  dim3 grid((L.N / KT) * (L.N / (2 * KT)), (nrhs + R - 1) / R);
  if (f) {
    if constexpr (std::is_same<Y, zdf>::value) {
      return WL_EINVAL;  // no residual form for double-float output
    } else {
      WL_TRY(set_smem_limit((const void *)k_stencil_tile<T, S, Y, R, 1>, smem, limit_set[1]));
      k_stencil_tile<T, S, Y, R, 1><<<grid, 256, smem, s>>>(L.geo, A, (const cx<T> *)x, (const Y *)f, (Y *)y, nrhs,
                                                             vec);
    }
  } else {
    WL_TRY(set_smem_limit((const void *)k_stencil_tile<T, S, Y, R, 0>, smem, limit_set[0]));
    k_stencil_tile<T, S, Y, R, 0><<<grid, 256, smem, s>>>(L.geo, A, (const cx<T> *)x, nullptr, (Y *)y, nrhs, vec);
  }
  return WL_OK;
}

// the tiled form for grids the tiling covers and batches of at least 8
template <typename T, typename S, typename Y>
static bool launch_stencil_tile(const Level &L, const S *A, const void *x, const void *f, void *y, int nrhs,
                                cudaStream_t s, int *rc) {
  if (L.N < 64 || L.N % (4 * KT) || nrhs < 8) return false;
  if constexpr (sizeof(T) == 4) {
    if (nrhs >= 32) {
      *rc = launch_stencil_tile_r<T, S, Y, 32>(L, A, x, f, y, nrhs, s);
      return true;
    }
  }
  if (nrhs >= 16) *rc = launch_stencil_tile_r<T, S, Y, 16>(L, A, x, f, y, nrhs, s);
  else *rc = launch_stencil_tile_r<T, S, Y, 8>(L, A, x, f, y, nrhs, s);
  return true;
}

int stencil_apply(wl_amg *a, int l, int prec, const void *x, void *y, const void *f, int nrhs,
                  cudaStream_t s) {
  const Level &L = a->lev[l];
  const LevelOps &o = ops_of(L, prec);
  long tot = (long)L.n * nrhs;
  unsigned grid = WL_GRID(tot, 256);
  wl_count_launches(1);
  int rc = WL_OK;
  if (prec == WL_FP64) {
    if (!launch_stencil_tile<double, zd, zd>(L, o.A.as<zd>(), x, f, y, nrhs, s, &rc))
      k_stencil<double, zd><<<grid, 256, 0, s>>>(L.geo, o.A.as<zd>(), (const zd *)x, (const zd *)f, (zd *)y, nrhs);
  } else if (prec == WL_FP32) {
    if (!launch_stencil_tile<float, zf, zf>(L, o.A.as<zf>(), x, f, y, nrhs, s, &rc))
      k_stencil<float, zf><<<grid, 256, 0, s>>>(L.geo, o.A.as<zf>(), (const zf *)x, (const zf *)f, (zf *)y, nrhs);
  } else {
    if (!launch_stencil_tile<float, zb, zf>(L, o.A.as<zb>(), x, f, y, nrhs, s, &rc))
      k_stencil<float, zb><<<grid, 256, 0, s>>>(L.geo, o.A.as<zb>(), (const zf *)x, (const zf *)f, (zf *)y, nrhs);
  }
  WL_TRY(rc);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

// block-resident sweeps of a small level: launch parameter RC | STAGE << 8
// (RC right-hand sides per block; STAGE = 1: stencil rows and denominators
// in shared memory too)
#define WL_BLOCK_SMEM_MAX (227 * 1024)
static size_t block_smem(const Level &L, int param, int prec) {
  int RC = param & 255;
  bool stage = (param >> 8) & 1;
  size_t ct = prec == WL_FP64 ? 16 : 8, t = ct / 2;
  size_t sz = prec == WL_FP64 ? 16 : (prec == WL_FP32 ? 8 : 4);
  return (size_t)L.n * 2 * RC * ct * 2 + (stage ? (size_t)L.n * 36 * sz + (size_t)L.n * 2 * t + 16 : 0);
}
static bool block_fits(const Level &L, int param, int prec) {
  return (param & 255) >= 1 && (param >> 9) == 0 && block_smem(L, param, prec) <= WL_BLOCK_SMEM_MAX;
}

template <typename T, typename S, bool STAGE>
static int launch_block_s(const Level &L, const LevelOps &o, int sweeps, void *x, void *r, int nrhs, double omega,
                          cudaStream_t s, int RC, size_t smem) {
  static std::atomic<unsigned long long> limit_set{0};
  WL_TRY(set_smem_limit((const void *)k_kacz_block<T, S, STAGE>, WL_BLOCK_SMEM_MAX, limit_set));
  long items = (long)(L.n >> 4) * RC;
  int nt = (int)std::min<long>(256, std::max<long>(32, (items + 31) / 32 * 32));
  k_kacz_block<T, S, STAGE><<<(nrhs + RC - 1) / RC, nt, smem, s>>>(L.geo, sweeps, RC, o.A.as<S>(), o.den.as<T>(),
                                                                  (cx<T> *)x, (cx<T> *)r, nrhs, (T)omega);
  return WL_OK;
}
template <typename T, typename S>
static int launch_block(const Level &L, const LevelOps &o, int sweeps, void *x, void *r, int nrhs, double omega,
                        cudaStream_t s, int param, int prec) {
  size_t smem = block_smem(L, param, prec);
  if ((param >> 8) & 1)
    return launch_block_s<T, S, true>(L, o, sweeps, x, r, nrhs, omega, s, param & 255, smem);
  return launch_block_s<T, S, false>(L, o, sweeps, x, r, nrhs, omega, s, param & 255, smem);
}

// tile-coloured launch for tile colour tc (one quarter of a sweep)
static bool tile_ok(int N) { return N >= 64 && N % (4 * KT) == 0; }

// shared memory of a tile block.  One right-hand side: all 64 stencil rows,
// denominators and r of tile + halo; several: r of tile + halo, denominators
// and the three-step ring of stencil rows
template <typename T, typename S>
static size_t tile_smem(int R) {
  size_t rows = R == 1 ? (size_t)KT * KT * 36 * sizeof(S) : (size_t)3 * 4 * 36 * sizeof(S);
  size_t index = R == 1 ? 0 : (size_t)KTH * KTH * sizeof(int);  // site-index table
  return rows + index + (size_t)KT * KT * 2 * sizeof(T) + (size_t)KTH * KTH * 2 * R * sizeof(cx<T>);
}

// 1 if a persistent tile launch on the current device reported a wait that ran
// out since the last call (the flag is cleared); read on stream s after it
int tile_timeout_take(cudaStream_t s) {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&v, g_tile_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return 0;
  if (v) {
    cudaMemcpyToSymbolAsync(g_tile_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    wl_set_error("a Kaczmarz tile launch ran out of time waiting for its own copies; results are not valid");
  }
  return v;
}

// shared memory of the persistent form: two r buffers, step scales, the
// stencil-row ring, the site-index table and two mbarriers
template <typename T, typename S>
static size_t tile_smem_p(int R) {
  return (size_t)2 * KTH * KTH * 2 * R * sizeof(cx<T>) + (size_t)KT * KT * 2 * sizeof(T) +
         (size_t)3 * 4 * 36 * sizeof(S) + (size_t)KTH * KTH * sizeof(int) + 8 + 2 * sizeof(uint64_t);
}

template <typename T, typename S, int R, int RPT, bool PAIRED>
static int launch_tile_p(const Level &L, const LevelOps &o, int tc, void *x, void *r, int nrhs, double omega,
                         cudaStream_t s) {
  size_t smem = tile_smem_p<T, S>(R);
  static std::atomic<unsigned long long> limit_set{0};
  WL_TRY(set_smem_limit((const void *)k_kacz_tile_p<T, S, R, RPT, PAIRED>, smem, limit_set));
  static std::atomic<int> per_sm{0};  // resident blocks per SM, from the occupancy calculator
  int nb = per_sm.load();
  if (nb == 0) {
    WL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_kacz_tile_p<T, S, R, RPT, PAIRED>, 4 * R / RPT,
                                                          smem));
    nb = std::max(nb, 1);
    per_sm.store(nb);
  }
  int dev = 0, nsm = 0;
  WL_CUDA(cudaGetDevice(&dev));
  WL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int ntiles = (L.N / (2 * KT)) * (L.N / (4 * KT));
  int nitems = ntiles * (nrhs / R);
  int grid = std::min(nitems, nb * nsm);
  k_kacz_tile_p<T, S, R, RPT, PAIRED><<<grid, 4 * R / RPT, smem, s>>>(L.geo, tc, o.A.as<S>(), o.den.as<T>(),
                                                                      (cx<T> *)x, (cx<T> *)r, nrhs, (T)omega,
                                                                      ntiles);
  return WL_OK;
}

// persistent form usable: full chunks, rows on 16-byte boundaries
template <typename T>
static bool tile_p_ok(const void *r, int nrhs, int R) {
  return ((uintptr_t)r % 16 == 0) && nrhs % R == 0 && (R * sizeof(cx<T>)) % 16 == 0 &&
         (nrhs * sizeof(cx<T>)) % 16 == 0;
}

template <typename T, typename S, int R, int RPT, bool PAIRED = false, bool SPLIT = false>
static int launch_tile_r(const Level &L, const LevelOps &o, int tc, void *x, void *r, int nrhs, double omega,
                         cudaStream_t s, bool persist = false) {
  if constexpr (!SPLIT) {
    if (persist && tile_p_ok<T>(r, nrhs, R))
      return launch_tile_p<T, S, R, RPT, PAIRED>(L, o, tc, x, r, nrhs, omega, s);
  }
  size_t smem = tile_smem<T, S>(R);
  static std::atomic<unsigned long long> limit_set{0};  // devices whose limit is raised
  WL_TRY(set_smem_limit((const void *)k_kacz_tile<T, S, R, RPT, PAIRED, SPLIT>, smem, limit_set));
  int vec = ((uintptr_t)r % 16 == 0) && (sizeof(T) == 8 || nrhs % 2 == 0);
  dim3 grid((L.N / (2 * KT)) * (L.N / (4 * KT)), (nrhs + R - 1) / R);
  constexpr int NT = SPLIT ? 8 * R : 4 * R / RPT;
  k_kacz_tile<T, S, R, RPT, PAIRED, SPLIT><<<grid, NT, smem, s>>>(L.geo, tc, o.A.as<S>(), o.den.as<T>(),
                                                                  (cx<T> *)x, (cx<T> *)r, nrhs, vec, (T)omega);
  return WL_OK;
}

// launch parameter of the tile kernel: R | RPT << 8 | P << 12 | Q << 13
// (right-hand-side chunk R, right-hand sides per thread RPT, 0 reading as 1,
// and 8 meaning one with paired FP32 FMAs; P = 1: the persistent form with
// double-buffered r, where the chunks are full and aligned, else the
// one-tile-per-block form; Q = 1 (FP32, RPT 8, P 0): each item split over a
// pair of lanes, tile_relax_split)
static inline int tile_param(int R, int rpt, int persist = 0, int split = 0) {
  return R | (rpt << 8) | (persist << 12) | (split << 13);
}

// default chunk: the smallest of 8, 16, 32 (FP64: 8, 16) that covers nrhs,
// so that few lanes idle and shared memory stays below 64 KB (FP32) or
// 90 KB (FP64) per block; one right-hand side per thread
static int tile_default_R(int nrhs, int prec) {
  if (nrhs <= 8) return 8;
  if (prec == WL_FP64 || nrhs <= 16) return 16;
  return 32;
}

template <typename T, typename S>
static int launch_tile(const Level &L, const LevelOps &o, int tc, void *x, void *r, int nrhs, double omega,
                       cudaStream_t s, int param) {
  if (nrhs == 1) {
    size_t smem = tile_smem<T, S>(1);
    k_kacz_tile1<T, S><<<(L.N / (2 * KT)) * (L.N / (4 * KT)), 128, smem, s>>>(
        L.geo, tc, o.A.as<S>(), o.den.as<T>(), (cx<T> *)x, (cx<T> *)r, (T)omega);
    return WL_OK;
  }
  int R = param & 255, rpt = std::max(1, (param >> 8) & 15);
  bool pe = (param >> 12) & 1, sp = (param >> 13) & 1;
  if constexpr (sizeof(T) == 8) {  // FP64: chunks up to 16, one right-hand side per thread
    if (R == 8) return launch_tile_r<T, S, 8, 1>(L, o, tc, x, r, nrhs, omega, s, pe);
    return launch_tile_r<T, S, 16, 1>(L, o, tc, x, r, nrhs, omega, s, pe);
  } else {  // rpt 8: one right-hand side per thread with paired FMAs
    bool pr = rpt == 8;
    if (sp) {  // each item over a pair of lanes
      if (R == 8) return launch_tile_r<T, S, 8, 1, true, true>(L, o, tc, x, r, nrhs, omega, s);
      if (R == 16) return launch_tile_r<T, S, 16, 1, true, true>(L, o, tc, x, r, nrhs, omega, s);
      return launch_tile_r<T, S, 32, 1, true, true>(L, o, tc, x, r, nrhs, omega, s);
    }
    if (R == 8)
      return pr ? launch_tile_r<T, S, 8, 1, true>(L, o, tc, x, r, nrhs, omega, s, pe)
                : launch_tile_r<T, S, 8, 1>(L, o, tc, x, r, nrhs, omega, s, pe);
    if (R == 16) {
      if (rpt == 2) return launch_tile_r<T, S, 16, 2>(L, o, tc, x, r, nrhs, omega, s, pe);
      return pr ? launch_tile_r<T, S, 16, 1, true>(L, o, tc, x, r, nrhs, omega, s, pe)
                : launch_tile_r<T, S, 16, 1>(L, o, tc, x, r, nrhs, omega, s, pe);
    }
    if (rpt == 2) return launch_tile_r<T, S, 32, 2>(L, o, tc, x, r, nrhs, omega, s, pe);
    return pr ? launch_tile_r<T, S, 32, 1, true>(L, o, tc, x, r, nrhs, omega, s, pe)
              : launch_tile_r<T, S, 32, 1>(L, o, tc, x, r, nrhs, omega, s, pe);
  }
}

int kaczmarz_tile(wl_amg *a, int l, int prec, void *x, void *r, int nrhs, int tc, cudaStream_t s, int R) {
  const Level &L = a->lev[l];
  if (!tile_ok(L.N)) return WL_EINVAL;
  const LevelOps &o = ops_of(L, prec);
  if (R <= 0) R = tile_param(tile_default_R(nrhs, prec), 1);
  wl_count_launches(1);
  if (prec == WL_FP64) return launch_tile<double, zd>(L, o, tc, x, r, nrhs, a->prm.omega, s, R);
  if (prec == WL_FP32) return launch_tile<float, zf>(L, o, tc, x, r, nrhs, a->prm.omega, s, R);
  return launch_tile<float, zb>(L, o, tc, x, r, nrhs, a->prm.omega, s, R);
}

static int coop_max_blocks(int prec) {
  return prec == WL_FP64 ? coop_blocks<double, zd>() : prec == WL_FP32 ? coop_blocks<float, zf>()
                                                                       : coop_blocks<float, zb>();
}

// blocks of 128 threads that cover one colour's work
static long colour_blocks(const Level &L, int nrhs) {
  long n16 = L.n >> 4;
  return WL_GRID(nrhs == 1 ? n16 * 32 : n16 * nrhs, 128);
}

static int run_sweeps(wl_amg *a, int l, int prec, void *x, void *r, int nrhs, int sweeps, const KTune &t,
                      cudaStream_t s) {
  const Level &L = a->lev[l];
  if (t.form == 2) {
    for (int sw = 0; sw < sweeps; ++sw)
      for (int tc = 0; tc < 4; ++tc) WL_TRY(kaczmarz_tile(a, l, prec, x, r, nrhs, tc, s, t.param));
  } else if (t.form == 1) {
    const LevelOps &o = ops_of(L, prec);
    wl_count_launches(1);
    int rc;
    if (prec == WL_FP64) rc = launch_coop<double, zd>(L, o, sweeps, x, r, nrhs, a->prm.omega, s, t.param);
    else if (prec == WL_FP32) rc = launch_coop<float, zf>(L, o, sweeps, x, r, nrhs, a->prm.omega, s, t.param);
    else rc = launch_coop<float, zb>(L, o, sweeps, x, r, nrhs, a->prm.omega, s, t.param);
    WL_TRY(rc);
  } else if (t.form == 3) {
    if (!block_fits(L, t.param, prec) || nrhs < 2) return WL_EINVAL;
    const LevelOps &o = ops_of(L, prec);
    wl_count_launches(1);
    int rc;
    if (prec == WL_FP64) rc = launch_block<double, zd>(L, o, sweeps, x, r, nrhs, a->prm.omega, s, t.param, prec);
    else if (prec == WL_FP32)
      rc = launch_block<float, zf>(L, o, sweeps, x, r, nrhs, a->prm.omega, s, t.param, prec);
    else rc = launch_block<float, zb>(L, o, sweeps, x, r, nrhs, a->prm.omega, s, t.param, prec);
    WL_TRY(rc);
  } else {
    for (int sw = 0; sw < sweeps; ++sw)
      for (int c = 0; c < 16; ++c) WL_TRY(kaczmarz_colour(a, l, prec, x, r, nrhs, c, s));
  }
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

// The sweep form for (level, nrhs, precision).  The ordering is the user's
// (kacz_order); within it every form computes the same numbers, so the
// choice only affects speed.  Order: an explicit sweep_kernel, else the
// autotuner's measured choice, else the heuristic (cooperative launch when
// one colour's work fits one wave of resident blocks).
KTune sweep_form_of(wl_amg *a, int l, int prec, int nrhs) {
  const Level &L = a->lev[l];
  KTune t{nrhs, prec, 0, 0, 0.f};
  bool tile = a->prm.kacz_order == 1 && tile_ok(L.N);
  if (a->prm.sweep_kernel == 0)
    for (const KTune &k : L.tune)
      if (k.nrhs == nrhs && k.prec == prec && (k.form == 2) == tile) return k;
  if (tile) {
    t.form = 2;
    t.param = tile_param(tile_default_R(nrhs, prec), 1);
    return t;
  }
  int maxb = coop_max_blocks(prec);
  long need = colour_blocks(L, nrhs);
  int mode = a->prm.sweep_kernel;
  if (mode == 2 || (mode == 0 && need <= maxb)) {
    t.form = 1;
    t.param = (int)std::min<long>(need, maxb);
  }
  return t;
}

int kaczmarz_sweeps(wl_amg *a, int l, int prec, void *x, void *r, int nrhs, int sweeps, cudaStream_t s) {
  if (sweeps <= 0) return WL_OK;
  return run_sweeps(a, l, prec, x, r, nrhs, sweeps, sweep_form_of(a, l, prec, nrhs), s);
}

// Autotuner: time every launch form of one sweep on each level (the level's
// own cycle buffers, whose contents the next cycle overwrites) and keep the
// fastest.  Candidates: per-colour launches and the cooperative launch at
// 1, 1/2 and 1/4 of the resident-block limit (colour order); right-hand-side
// chunks 8, 16, 32 (tile order).  Runs outside stream capture, once per
// (nrhs, precision); sweep_kernel != 0 disables it.
int autotune_sweeps(wl_amg *a, int nrhs, int prec, cudaStream_t s) {
  if (a->prm.sweep_kernel != 0 || nrhs > a->cap) return WL_OK;
  cudaEvent_t e0, e1;
  WL_CUDA(cudaEventCreate(&e0));
  WL_CUDA(cudaEventCreate(&e1));
  int rc = WL_OK;
  for (int l = 0; l < a->L - 1 && rc == WL_OK; ++l) {
    Level &L = a->lev[l];
    bool tile = a->prm.kacz_order == 1 && tile_ok(L.N);
    bool have = false;
    for (const KTune &k : L.tune)
      if (k.nrhs == nrhs && k.prec == prec && (k.form == 2) == tile) have = true;
    if (have) continue;
    std::vector<KTune> cand;
    if (tile) {
      if (nrhs == 1) cand.push_back(KTune{nrhs, prec, 2, 1, 0.f});
      else
        for (int R : {8, 16, 32}) {
          if (prec == WL_FP64 && R > 16) continue;
          if (R / 2 >= nrhs && R > 8) continue;  // mostly idle lanes
          cand.push_back(KTune{nrhs, prec, 2, tile_param(R, 1), 0.f});
          if (prec != WL_FP64) cand.push_back(KTune{nrhs, prec, 2, tile_param(R, 8), 0.f});  // paired FMAs
          if (R >= 16 && prec != WL_FP64) cand.push_back(KTune{nrhs, prec, 2, tile_param(R, 2), 0.f});
          if (nrhs % R == 0) {  // persistent form (double-buffered r) where the chunks are full
            cand.push_back(KTune{nrhs, prec, 2, tile_param(R, 1, 1), 0.f});
            if (prec != WL_FP64) cand.push_back(KTune{nrhs, prec, 2, tile_param(R, 8, 1), 0.f});
          }
          if (prec != WL_FP64) cand.push_back(KTune{nrhs, prec, 2, tile_param(R, 8, 0, 1), 0.f});  // split pairs
        }
    } else {
      cand.push_back(KTune{nrhs, prec, 0, 0, 0.f});
      if (nrhs > 1)  // block-resident sweeps (thread per item, as forms 0 and 1 at nrhs > 1)
        for (int RC : {1, 2, 4, 8})
          for (int stage : {0, 1})  // stencil rows through the cache, or staged in shared memory
            if (RC <= nrhs && block_fits(L, RC | stage << 8, prec))
              cand.push_back(KTune{nrhs, prec, 3, RC | stage << 8, 0.f});
      int maxb = coop_max_blocks(prec);
      long need = colour_blocks(L, nrhs);
      if (need <= 4L * maxb)
        for (int div : {1, 2, 4}) {
          int b = (int)std::min<long>(need, std::max(1, maxb / div));
          bool dup = false;
          for (const KTune &c : cand) dup |= (c.form == 1 && c.param == b);
          if (!dup) cand.push_back(KTune{nrhs, prec, 1, b, 0.f});
        }
    }
    KTune best = cand[0];
    float best_us = 1e30f;
    for (KTune &c : cand) {
      rc = run_sweeps(a, l, prec, L.x.p, L.r.p, nrhs, 1, c, s);  // warm-up
      if (rc) break;
      if ((rc = (cudaEventRecord(e0, s) == cudaSuccess) ? WL_OK : WL_ECUDA)) break;
      for (int rep = 0; rep < 3 && rc == WL_OK; ++rep) rc = run_sweeps(a, l, prec, L.x.p, L.r.p, nrhs, 1, c, s);
      if (rc) break;
      float ms = 0;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = WL_ECUDA;
        break;
      }
      c.us = ms * 1e3f / 3;
      if (c.us < best_us) {
        best_us = c.us;
        best = c;
      }
    }
    if (rc == WL_OK) L.tune.push_back(best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == WL_ECUDA) wl_set_error("autotune_sweeps: CUDA error while timing");
  return rc;
}

// y = A_0 x in FP32 arithmetic from the FP32 copy of the level-0 stencil
// (Dhat), x float, y widened to double or stored as a double-float with a
// zero low part: the Arnoldi matvec of an FP32 cycle
template <typename Y>
static int stencil_apply32_to(wl_amg *a, const void *x, Y *y, int nrhs, cudaStream_t s) {
  const Level &L = a->lev[0];
  long tot = (long)L.n * nrhs;
  wl_count_launches(1);
  int rc = WL_OK;
  if (!launch_stencil_tile<float, zf, Y>(L, L.op32.A.as<zf>(), x, nullptr, y, nrhs, s, &rc))
    k_stencil<float, zf, Y><<<WL_GRID(tot, 256), 256, 0, s>>>(L.geo, L.op32.A.as<zf>(), (const zf *)x, nullptr, y,
                                                              nrhs);
  WL_TRY(rc);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}
int stencil_apply32_to64(wl_amg *a, const void *x, zd *y, int nrhs, cudaStream_t s) {
  return stencil_apply32_to<zd>(a, x, y, nrhs, s);
}
int stencil_apply32_to_df(wl_amg *a, const void *x, zdf *y, int nrhs, cudaStream_t s) {
  return stencil_apply32_to<zdf>(a, x, y, nrhs, s);
}

int restrict_op(wl_amg *a, int l, int prec, const void *r, void *fc, int nrhs, cudaStream_t s) {
  const Level &F = a->lev[l], &Cl = a->lev[l + 1];
  const LevelOps &o = ops_of(F, prec);
  int lgB = ilog2(F.B);
  long tot = (long)Cl.n * nrhs;
  unsigned grid = WL_GRID(tot, 128);
  wl_count_launches(1);
  if (prec == WL_FP64)
    k_restrict<double, zd><<<grid, 128, 0, s>>>(F.geo, Cl.geo, lgB, o.P.as<zd>(), (const zd *)r, (zd *)fc, nrhs);
  else if (prec == WL_FP32)
    k_restrict<float, zf><<<grid, 128, 0, s>>>(F.geo, Cl.geo, lgB, o.P.as<zf>(), (const zf *)r, (zf *)fc, nrhs);
  else
    k_restrict<float, zb><<<grid, 128, 0, s>>>(F.geo, Cl.geo, lgB, o.P.as<zb>(), (const zf *)r, (zf *)fc, nrhs);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

int prolong_op(wl_amg *a, int l, int prec, const void *e, void *x, int nrhs, cudaStream_t s) {
  const Level &F = a->lev[l], &Cl = a->lev[l + 1];
  const LevelOps &o = ops_of(F, prec);
  int lgB = ilog2(F.B);
  long tot = (long)F.n * nrhs;
  unsigned grid = WL_GRID(tot, 256);
  wl_count_launches(1);
  if (prec == WL_FP64)
    k_prolong<double, zd><<<grid, 256, 0, s>>>(F.geo, Cl.geo, lgB, o.P.as<zd>(), (const zd *)e, (zd *)x, nrhs);
  else if (prec == WL_FP32)
    k_prolong<float, zf><<<grid, 256, 0, s>>>(F.geo, Cl.geo, lgB, o.P.as<zf>(), (const zf *)e, (zf *)x, nrhs);
  else
    k_prolong<float, zb><<<grid, 256, 0, s>>>(F.geo, Cl.geo, lgB, o.P.as<zb>(), (const zf *)e, (zf *)x, nrhs);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

int coarsest_apply(wl_amg *a, int prec, const void *f, void *x, int nrhs, cudaStream_t s) {
  dim3 grid(WL_GRID(a->nc, 8), nrhs);
  wl_count_launches(1);
  if (prec == WL_FP64)
    k_coarsest<double><<<grid, 256, 0, s>>>(a->nc, a->Ainv.as<zd>(), (const zd *)f, (zd *)x, nrhs);
  else
    k_coarsest<float><<<grid, 256, 0, s>>>(a->nc, a->Ainv.as<zd>(), (const zf *)f, (zf *)x, nrhs);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

// recursive cycle on level l: lev[l].x = M(lev[l].f) starting from x = 0
static int cycle_level(wl_amg *a, int l, int nrhs, int prec, cudaStream_t s) {
  Level &L = a->lev[l];
  size_t eb = prec_bytes(prec);
  size_t vb = eb * (size_t)L.n * 2 * nrhs;
  if (l == a->L - 1) return coarsest_apply(a, prec, L.f.p, L.x.p, nrhs, s);
  WL_CUDA(cudaMemsetAsync(L.x.p, 0, vb, s));
  WL_CUDA(cudaMemcpyAsync(L.r.p, L.f.p, vb, cudaMemcpyDeviceToDevice, s));
  WL_TRY(kaczmarz_sweeps(a, l, prec, L.x.p, L.r.p, nrhs, a->prm.nu_pre, s));
  Level &C = a->lev[l + 1];
  WL_TRY(restrict_op(a, l, prec, L.r.p, C.f.p, nrhs, s));
  int gamma = (a->prm.cycle == WL_CYCLE_W) ? 2 : 1;
  size_t cb = eb * (size_t)C.n * 2 * nrhs;
  for (int g = 0; g < gamma; ++g) {
    if (g > 0) {
      // coarse residual of the correction so far, then one more cycle
      WL_CUDA(cudaMemcpyAsync(C.t.p, C.x.p, cb, cudaMemcpyDeviceToDevice, s));
      WL_TRY(stencil_apply(a, l + 1, prec, C.t.p, C.f.p, C.f.p, nrhs, s));
    }
    WL_TRY(cycle_level(a, l + 1, nrhs, prec, s));
    if (g > 0) {
      long ne = (long)C.n * 2 * nrhs;
      wl_count_launches(1);
      if (prec == WL_FP64) k_axpy_inplace<double><<<WL_GRID(ne, 256), 256, 0, s>>>(C.x.as<zd>(), C.t.as<zd>(), ne);
      else k_axpy_inplace<float><<<WL_GRID(ne, 256), 256, 0, s>>>(C.x.as<zf>(), C.t.as<zf>(), ne);
      WL_CUDA(cudaGetLastError());
    }
  }
  WL_TRY(prolong_op(a, l, prec, C.x.p, L.x.p, nrhs, s));
  WL_TRY(stencil_apply(a, l, prec, L.x.p, L.r.p, L.f.p, nrhs, s));
  WL_TRY(kaczmarz_sweeps(a, l, prec, L.x.p, L.r.p, nrhs, a->prm.nu_post, s));
  return WL_OK;
}

// lev[0].x = M(lev[0].f) without graph capture (setup's adaptive step)
int cycle_direct(wl_amg *a, int nrhs, int prec, cudaStream_t s) { return cycle_level(a, 0, nrhs, prec, s); }

// lev[0].x = M(lev[0].f); captured once per (nrhs, precision) as a CUDA graph
// Capture and instantiate the cycle graph for (nrhs, prec) unless it exists;
// nothing is launched.  A capture in progress forbids device-wide
// synchronisation anywhere in the process, so callers that run beside other
// threads (the serving workers) capture every width they need up front.
int cycle_prepare(wl_amg *a, int nrhs, int prec, cudaStream_t s, const wl_amg::G **out) {
  for (auto &g : a->graphs)
    if (g.nrhs == nrhs && g.prec == prec) {
      if (out) *out = &g;
      return WL_OK;
    }
  WL_TRY(autotune_sweeps(a, nrhs, prec, s));  // measured launch forms, before the capture
  cudaGraph_t graph;
  long long before = wl_launch_count();
  WL_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = cycle_level(a, 0, nrhs, prec, s);
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  long long kernels = wl_launch_count() - before;  // captured, not run
  wl_count_launches(-kernels);
  if (rc) {
    if (e == cudaSuccess) cudaGraphDestroy(graph);
    return rc;
  }
  WL_CUDA(e);
  wl_amg::G gg;
  gg.nrhs = nrhs;
  gg.prec = prec;
  gg.kernels = kernels;
  e = cudaGraphInstantiate(&gg.exec, graph, 0);
  cudaGraphDestroy(graph);
  WL_CUDA(e);
  a->graphs.push_back(gg);
  if (out) *out = &a->graphs.back();
  return WL_OK;
}

int cycle_run(wl_amg *a, int nrhs, int prec, cudaStream_t s) {
  const wl_amg::G *g = nullptr;
  WL_TRY(cycle_prepare(a, nrhs, prec, s, &g));
  WL_CUDA(cudaGraphLaunch(g->exec, s));
  wl_count_launches(g->kernels);
  return WL_OK;
}

}  // namespace wl

// ------------------------------------------------------ per-step entry points
static int check_amg(wl_amg *a, int level, int nrhs, int prec, const char *who) {
  if (!a || nrhs < 1 || level < 0 || level >= a->L ||
      (prec != WL_FP64 && prec != WL_FP32 && prec != WL_FP32_BF16)) {
    wl_set_error("%s: invalid argument", who);
    return WL_EINVAL;
  }
  return wl::enter(a->op);
}

struct StepBufs {
  DBuf b[3];
  ~StepBufs() {
    for (auto &x : b) x.release();
  }
};

extern "C" int amg_level_apply(wl_amg *a, int level, const void *x, void *y, int nrhs, int prec) {
  WL_TRY(check_amg(a, level, nrhs, prec, "amg_level_apply"));
  if (!x || !y) return WL_EINVAL;
  cudaStream_t s = a->op->stream;
  int n2 = a->lev[level].n * 2;
  size_t vb = wl::prec_bytes(prec) * (size_t)n2 * nrhs;
  int pin = prec == WL_FP64 ? WL_FP64 : WL_FP32;
  StepBufs sb;
  WL_TRY(sb.b[0].alloc(vb));
  WL_TRY(sb.b[1].alloc(vb));
  WL_TRY(wl::to_internal((const zd *)x, sb.b[0].p, n2, nrhs, pin, s));
  WL_TRY(wl::stencil_apply(a, level, prec, sb.b[0].p, sb.b[1].p, nullptr, nrhs, s));
  WL_TRY(wl::from_internal(sb.b[1].p, (zd *)y, n2, nrhs, pin, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

// does launch form (form, param) exist for a sweep of `level` (not the
// coarsest) with nrhs right-hand sides in precision prec?
static bool form_exists(const wl_amg *a, int level, int nrhs, int prec, int form, int param) {
  const Level &L = a->lev[level];
  bool tile = a->prm.kacz_order == 1 && wl::tile_ok(L.N);
  int R = param & 255, rpt = std::max(1, (param >> 8) & 15);
  if (param >> 14) return false;
  if ((param >> 13) & 1)  // split pairs: FP32, paired FMAs, one tile per block
    return tile && form == 2 && nrhs > 1 && prec != WL_FP64 && rpt == 8 && !((param >> 12) & 1) &&
           (R == 8 || R == 16 || R == 32);
  return tile ? (form == 2 &&
                 (nrhs == 1 || (R == 8 && (rpt == 1 || rpt == 8)) ||
                  ((R == 16 || R == 32) && (rpt <= 2 || rpt == 8))) &&
                 !(prec == WL_FP64 && (R > 16 || rpt > 1)))
              : ((form == 0) || (form == 1 && param >= 1) ||
                 (form == 3 && nrhs > 1 && wl::block_fits(L, param, prec)));
}

// form < 0: the solver's own choice; else an explicit launch form (KTune)
static int kaczmarz_entry(wl_amg *a, int level, void *x, void *r, int nrhs, int sweeps, int prec, int form,
                          int param, const char *who) {
  WL_TRY(check_amg(a, level, nrhs, prec, who));
  if (!x || !r || sweeps < 0 || level == a->L - 1) {
    wl_set_error("%s: invalid argument (the coarsest level is not relaxed)", who);
    return WL_EINVAL;
  }
  if (form >= 0 && !form_exists(a, level, nrhs, prec, form, param)) {
    wl_set_error("%s: launch form %d / %d does not exist for this level and ordering", who, form, param);
    return WL_EINVAL;
  }
  cudaStream_t s = a->op->stream;
  int n2 = a->lev[level].n * 2;
  size_t vb = wl::prec_bytes(prec) * (size_t)n2 * nrhs;
  int pin = prec == WL_FP64 ? WL_FP64 : WL_FP32;
  StepBufs sb;
  WL_TRY(sb.b[0].alloc(vb));
  WL_TRY(sb.b[1].alloc(vb));
  WL_TRY(wl::to_internal((const zd *)x, sb.b[0].p, n2, nrhs, pin, s));
  WL_TRY(wl::to_internal((const zd *)r, sb.b[1].p, n2, nrhs, pin, s));
  if (form < 0) {
    WL_TRY(wl::kaczmarz_sweeps(a, level, prec, sb.b[0].p, sb.b[1].p, nrhs, sweeps, s));
  } else if (sweeps > 0) {
    KTune t{nrhs, prec, form, param, 0.f};
    WL_TRY(wl::run_sweeps(a, level, prec, sb.b[0].p, sb.b[1].p, nrhs, sweeps, t, s));
  }
  WL_TRY(wl::from_internal(sb.b[0].p, (zd *)x, n2, nrhs, pin, s));
  WL_TRY(wl::from_internal(sb.b[1].p, (zd *)r, n2, nrhs, pin, s));
  WL_CUDA(cudaStreamSynchronize(s));
  if (wl::tile_timeout_take(s)) return WL_TIMEOUT;
  return WL_OK;
}

extern "C" int amg_kaczmarz(wl_amg *a, int level, void *x, void *r, int nrhs, int sweeps, int prec) {
  return kaczmarz_entry(a, level, x, r, nrhs, sweeps, prec, -1, 0, "amg_kaczmarz");
}

extern "C" int amg_kaczmarz_form(wl_amg *a, int level, void *x, void *r, int nrhs, int sweeps, int prec, int form,
                                 int param) {
  if (form < 0) {
    wl_set_error("amg_kaczmarz_form: form must be 0, 1 or 2");
    return WL_EINVAL;
  }
  return kaczmarz_entry(a, level, x, r, nrhs, sweeps, prec, form, param, "amg_kaczmarz_form");
}

extern "C" int amg_restrict(wl_amg *a, int level, const void *r, void *fc, int nrhs, int prec) {
  WL_TRY(check_amg(a, level, nrhs, prec, "amg_restrict"));
  if (!r || !fc || level == a->L - 1) return WL_EINVAL;
  cudaStream_t s = a->op->stream;
  int nf2 = a->lev[level].n * 2, nc2 = a->lev[level + 1].n * 2;
  size_t eb = wl::prec_bytes(prec);
  int pin = prec == WL_FP64 ? WL_FP64 : WL_FP32;
  StepBufs sb;
  WL_TRY(sb.b[0].alloc(eb * nf2 * nrhs));
  WL_TRY(sb.b[1].alloc(eb * nc2 * nrhs));
  WL_TRY(wl::to_internal((const zd *)r, sb.b[0].p, nf2, nrhs, pin, s));
  WL_TRY(wl::restrict_op(a, level, prec, sb.b[0].p, sb.b[1].p, nrhs, s));
  WL_TRY(wl::from_internal(sb.b[1].p, (zd *)fc, nc2, nrhs, pin, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

extern "C" int amg_prolong(wl_amg *a, int level, const void *e, void *x, int nrhs, int prec) {
  WL_TRY(check_amg(a, level, nrhs, prec, "amg_prolong"));
  if (!e || !x || level == a->L - 1) return WL_EINVAL;
  cudaStream_t s = a->op->stream;
  int nf2 = a->lev[level].n * 2, nc2 = a->lev[level + 1].n * 2;
  size_t eb = wl::prec_bytes(prec);
  int pin = prec == WL_FP64 ? WL_FP64 : WL_FP32;
  StepBufs sb;
  WL_TRY(sb.b[0].alloc(eb * nc2 * nrhs));
  WL_TRY(sb.b[1].alloc(eb * nf2 * nrhs));
  WL_TRY(wl::to_internal((const zd *)e, sb.b[0].p, nc2, nrhs, pin, s));
  WL_TRY(wl::to_internal((const zd *)x, sb.b[1].p, nf2, nrhs, pin, s));
  WL_TRY(wl::prolong_op(a, level, prec, sb.b[0].p, sb.b[1].p, nrhs, s));
  WL_TRY(wl::from_internal(sb.b[1].p, (zd *)x, nf2, nrhs, pin, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

extern "C" int amg_coarsest(wl_amg *a, const void *f, void *x, int nrhs) {
  WL_TRY(check_amg(a, 0, nrhs, WL_FP64, "amg_coarsest"));
  if (!f || !x) return WL_EINVAL;
  cudaStream_t s = a->op->stream;
  StepBufs sb;
  WL_TRY(sb.b[0].alloc(sizeof(zd) * a->nc * nrhs));
  WL_TRY(sb.b[1].alloc(sizeof(zd) * a->nc * nrhs));
  WL_TRY(wl::to_internal((const zd *)f, sb.b[0].p, a->nc, nrhs, WL_FP64, s));
  WL_TRY(wl::coarsest_apply(a, WL_FP64, sb.b[0].p, sb.b[1].p, nrhs, s));
  WL_TRY(wl::from_internal(sb.b[1].p, (zd *)x, a->nc, nrhs, WL_FP64, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

extern "C" int amg_cycle(wl_amg *a, const void *f, void *x, int nrhs, int prec) {
  WL_TRY(check_amg(a, 0, nrhs, prec, "amg_cycle"));
  if (!f || !x) return WL_EINVAL;
  WL_TRY(wl::ensure_workspace(a, nrhs, prec));
  cudaStream_t s = a->op->stream;
  int n2 = a->lev[0].n * 2;
  int pin = prec == WL_FP64 ? WL_FP64 : WL_FP32;
  WL_TRY(wl::to_internal((const zd *)f, a->lev[0].f.p, n2, nrhs, pin, s));
  WL_TRY(wl::cycle_run(a, nrhs, prec, s));
  WL_TRY(wl::from_internal(a->lev[0].x.p, (zd *)x, n2, nrhs, pin, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

extern "C" int amg_pin_sweep_form(wl_amg *a, int level, int nrhs, int prec, int form, int param) {
  WL_TRY(check_amg(a, level, nrhs, prec, "amg_pin_sweep_form"));
  if (level == a->L - 1 || !form_exists(a, level, nrhs, prec, form, param)) {
    wl_set_error("amg_pin_sweep_form: launch form %d / %d does not exist for this level and ordering", form, param);
    return WL_EINVAL;
  }
  std::vector<KTune> &tv = a->lev[level].tune;
  for (KTune &k : tv)
    if (k.nrhs == nrhs && k.prec == prec) {
      k = KTune{nrhs, prec, form, param, 0.f};
      return WL_OK;
    }
  tv.push_back(KTune{nrhs, prec, form, param, 0.f});
  return WL_OK;
}

extern "C" int amg_sweep_form(wl_amg *a, int level, int nrhs, int prec, int *form, int *param, float *us) {
  if (!a || !form || !param || !us || level < 0 || level >= a->L - 1 || nrhs < 1 ||
      (prec != WL_FP64 && prec != WL_FP32 && prec != WL_FP32_BF16)) {
    wl_set_error("amg_sweep_form: invalid argument");
    return WL_EINVAL;
  }
  KTune t = wl::sweep_form_of(a, level, prec, nrhs);
  *form = t.form;
  *param = t.param;
  *us = t.us;
  return WL_OK;
}
