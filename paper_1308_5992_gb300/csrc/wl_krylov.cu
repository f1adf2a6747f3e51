// wl_krylov.cu -- flexible GMRES(m) (Saad 1993) around the AMG cycle,
// batched over right-hand sides in lock step: right preconditioning
// z_j = M(v_j) (Sec. 4 uses GMRES(32) with a W(4,4) cycle), classical
// Gram-Schmidt with optional reorthogonalisation in FP64 or in double-float
// on the FP32 pipes, per right-hand-side Givens rotations in FP64, restarts
// that recompute the true residual in FP64 (iterative refinement when the
// cycle runs in FP32), the two-step Schur solve of Sec. 3.2 around it
// (amg_solve, amg_solve_host), and the batch as one or two concurrent
// solve lanes.
#include <math.h>
#include <cmath>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "wl_common.cuh"

namespace wl {
int eo_reduce_internal(wl_op *op, const zd *b, zd *bh, int nrhs, cudaStream_t s);
int eo_reconstruct_internal(wl_op *op, const zd *b, const zd *xe, zd *psi, int nrhs, cudaStream_t s);
int take_even_internal(wl_op *op, const zd *psi, zd *xe, int nrhs, cudaStream_t s);
int resolve_levels(int N, amg_params *p, int *Nl);
}

// per right-hand-side Krylov scalars
struct KS {
  int m, nrhs;
  zd *hcol;    // [nrhs][m+1] accumulated column of H
  zd *hpass;   // [m+1][nrhs] coefficients of the current Gram-Schmidt pass (rhs innermost)
  zd *H;       // [nrhs][m+1][m]
  zd *g;       // [nrhs][m+1]
  zd *cs;      // [nrhs][m]
  double *cc;  // [nrhs][m]
  zd *y;       // [nrhs][m]
  zd *yT;      // [m][nrhs] the same, rhs innermost
  double *bnorm, *beta, *nrm2, *inv;  // [nrhs]
  int *active, *stop, *jend, *iters;  // [nrhs]
  int *nanf;                          // [nrhs] non-finite value seen (Arnoldi residual, or masked input)
  int *running;                       // [1]
  float4 *hpd;   // [m+1][nrhs][2] the coefficients of hpass as double-floats, for k_maxpy_df
  float2 *invdf; // [nrhs] inv as a double-float (hi, lo)
};

static KS ks_layout(void *base, int m, int nrhs) {
  KS k;
  k.m = m;
  k.nrhs = nrhs;
  char *p = (char *)base;
  auto take = [&](size_t bytes) {
    char *q = p;
    p += (bytes + 255) & ~(size_t)255;
    return q;
  };
  k.hcol = (zd *)take(sizeof(zd) * nrhs * (m + 1));
  k.hpass = (zd *)take(sizeof(zd) * nrhs * (m + 1));
  k.H = (zd *)take(sizeof(zd) * nrhs * (m + 1) * m);
  k.g = (zd *)take(sizeof(zd) * nrhs * (m + 1));
  k.cs = (zd *)take(sizeof(zd) * nrhs * m);
  k.cc = (double *)take(sizeof(double) * nrhs * m);
  k.y = (zd *)take(sizeof(zd) * nrhs * m);
  k.yT = (zd *)take(sizeof(zd) * nrhs * m);
  k.bnorm = (double *)take(sizeof(double) * nrhs);
  k.beta = (double *)take(sizeof(double) * nrhs);
  k.nrm2 = (double *)take(sizeof(double) * nrhs);
  k.inv = (double *)take(sizeof(double) * nrhs);
  k.active = (int *)take(sizeof(int) * nrhs);
  k.stop = (int *)take(sizeof(int) * nrhs);
  k.jend = (int *)take(sizeof(int) * nrhs);
  k.iters = (int *)take(sizeof(int) * nrhs);
  k.nanf = (int *)take(sizeof(int) * nrhs);
  k.running = (int *)take(sizeof(int) * 4);
  k.hpd = (float4 *)take(sizeof(float4) * 2 * nrhs * (m + 1));
  k.invdf = (float2 *)take(sizeof(float2) * nrhs);
  return k;
}

// ------------------------------------------------------------- reductions
// Block layout: blockDim = R * G with R = nrhs (<= 256) and G a power of two;
// thread t handles right-hand side t % R, so element e of a vector
// ([n][2][nrhs] flattened) always belongs to rhs e % R.
#define KCH 12  // dots per launch
// KC (the number of dots) is a template parameter: predicated-off FP64
// FMAs still occupy the FP64 pipe, so a run-time count would cost every
// launch the work of KCH dots
template <typename Tv, int KC>
__global__ void k_mdot(const cx<Tv> *__restrict__ V, long vstride, const zd *__restrict__ w, long E, int R,
                       zd *__restrict__ part) {
  extern __shared__ unsigned char sm_raw[];
  zd *sm = (zd *)sm_raw;  // [KC][blockDim]
  int t = threadIdx.x, nt = blockDim.x;
  int G = nt / R, q = t / R;
  zd acc[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) acc[k] = mk(0.0, 0.0);
  long stride = (long)gridDim.x * nt;
  for (long e = (long)blockIdx.x * nt + t; e < E; e += stride) {
    zd we = w[e];
    zd v[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) v[k] = ccast<double>(V[k * vstride + e]);
#pragma unroll
    for (int k = 0; k < KC; ++k) cfmac(acc[k], v[k], we);
  }
#pragma unroll
  for (int k = 0; k < KC; ++k) sm[k * nt + t] = acc[k];
  __syncthreads();
  for (int s = G >> 1; s > 0; s >>= 1) {
    if (q < s)
#pragma unroll
      for (int k = 0; k < KC; ++k) sm[k * nt + t] = sm[k * nt + t] + sm[k * nt + t + s * R];
    __syncthreads();
  }
  if (q == 0)
#pragma unroll
    for (int k = 0; k < KC; ++k) part[((long)blockIdx.x * KC + k) * R + t] = sm[k * nt + t];
}

// |w_r|^2 per right-hand side in the layout of k_mdot with one dot: only the
// real part is accumulated (two FMAs per complex element instead of four;
// the same roundings as the real part of conj(w) w)
__global__ void k_norm2(const zd *__restrict__ w, long E, int R, zd *__restrict__ part) {
  extern __shared__ unsigned char sm_raw[];
  double *sm = (double *)sm_raw;  // [blockDim]
  int t = threadIdx.x, nt = blockDim.x;
  int G = nt / R, q = t / R;
  double acc = 0;
  long stride = (long)gridDim.x * nt;
  for (long e = (long)blockIdx.x * nt + t; e < E; e += stride) {
    zd we = w[e];
    acc = fma(we.re, we.re, acc);
    acc = fma(we.im, we.im, acc);
  }
  sm[t] = acc;
  __syncthreads();
  for (int s = G >> 1; s > 0; s >>= 1) {
    if (q < s) sm[t] = sm[t] + sm[t + s * R];
    __syncthreads();
  }
  if (q == 0) part[(long)blockIdx.x * R + t] = mk(sm[t], 0.0);
}

template <typename Tv>
static void launch_mdot(int kc, int nblk, int nt, size_t sm, cudaStream_t s, const cx<Tv> *V, long vstride,
                        const zd *w, long E, int R, zd *part) {
  switch (kc) {
#define WL_MDOT(K) \
  case K: k_mdot<Tv, K><<<nblk, nt, sm, s>>>(V, vstride, w, E, R, part); break;
    WL_MDOT(1) WL_MDOT(2) WL_MDOT(3) WL_MDOT(4) WL_MDOT(5) WL_MDOT(6)
    WL_MDOT(7) WL_MDOT(8) WL_MDOT(9) WL_MDOT(10) WL_MDOT(11) WL_MDOT(12)
#undef WL_MDOT
    default: break;
  }
}

// out[r][k0 + k] (= or +=) sum over blocks of part[b][k][r]: one warp per
// (k, r), lanes stride the blocks, shuffle tree (fixed order: deterministic)
__global__ void k_mdot_final(const zd *__restrict__ part, int nblk, int kc, int R, zd *out, int ostride,
                             int k0, int accumulate, zd *copy_to) {
  int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= kc * R) return;
  int k = wid / R, r = wid % R;
  zd s = mk(0.0, 0.0);
  for (int b = lane; b < nblk; b += 32) s = s + part[((long)b * kc + k) * R + r];
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    s.re += __shfl_down_sync(0xffffffffu, s.re, off);
    s.im += __shfl_down_sync(0xffffffffu, s.im, off);
  }
  if (lane) return;
  zd *o = out + (long)r * ostride + k0 + k;
  if (copy_to) copy_to[(long)(k0 + k) * R + r] = s;  // rhs innermost
  *o = accumulate ? (*o + s) : s;
}

// w += sign * sum_k V_k * coef[k][r]   (coef row stride cstride, rhs
// innermost so a warp's coefficient loads are contiguous); the
// k loop is unrolled by 4 with the four loads issued before the FMAs
template <typename Tv, int NEG>
__global__ void __launch_bounds__(256) k_maxpy(const cx<Tv> *__restrict__ V, long vstride, int kc,
                                               const zd *__restrict__ coef, int cstride, zd *__restrict__ w,
                                               long E, int R) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int r = (int)(e % R);
  const zd *cr = coef + r;
  zd acc = w[e];
  int k = 0;
  for (; k + 4 <= kc; k += 4) {
    zd v[4], c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = widen<double>(V[(k + u) * vstride + e]);
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = cr[(long)(k + u) * cstride];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (NEG) cfms(acc, c[u], v[u]);
      else cfma(acc, c[u], v[u]);
    }
  }
  for (; k < kc; ++k) {
    zd c = cr[(long)k * cstride];
    zd v = widen<double>(V[k * vstride + e]);
    if (NEG) cfms(acc, c, v);
    else cfma(acc, c, v);
  }
  w[e] = acc;
}

// out = f[rhs] in (the next Arnoldi vector) and its copy in the cycle
// precision, the next cycle's input (the cast rounds as k_cast does)
template <typename Tc>
__global__ void k_scale_rhs_cyc(const zd *__restrict__ in, zd *__restrict__ out, cx<Tc> *__restrict__ cyc,
                                const double *__restrict__ f, long E, int R) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  zd v = f[e % R] * in[e];
  out[e] = v;
  cyc[e] = ccast<Tc>(v);
}


__global__ void k_sub(const zd *__restrict__ a, const zd *__restrict__ b, zd *__restrict__ c, long E) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < E) c[e] = a[e] - b[e];
}

template <typename To, typename Ti>
__global__ void k_cast(const cx<Ti> *__restrict__ a, cx<To> *__restrict__ b, long E) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < E) b[e] = ccast<To>(a[e]);
}

// ------------------------------------------------ double-float Gram-Schmidt
// With amg_params.gs_arith = 1 the Krylov vectors v_j and w are zdf (hi + lo
// pairs of complex floats) and the Gram-Schmidt dots, updates and norms run
// on the FP32 pipes, whose rate on this GPU is 64 times the FP64 rate.  The
// arithmetic is built from two error-free transformations, applied to the
// (re, im) components of a pair at once through the paired round-to-nearest
// intrinsics (which the compiler never contracts into other operations):
//   two_sum (Knuth):  s + e = a + b exactly, six additions;
//   two_prod (FMA):   p + e = a * b exactly, e = fma(a, b, -p).
// A product of double-floats keeps hi * hi exactly and the cross terms
// hi * lo + lo * hi in FP32 (lo * lo, below 2^-48 of the product, is
// dropped); a running sum is a pair (s, c) renormalised after every step
// (|c| <= ulp(s) / 2).  Every step is exact to about 2^-47 of its result,
// against 2^-53 for FP64.

__host__ __device__ __forceinline__ float2 split_df(double v) {
  float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }

struct DF2 {
  float2 s, c;  // the value s + c, per component
};

// s + e = a + b exactly
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
  s = add2(a, b);
  float2 bv = sub2(s, a);
  float2 av = sub2(s, bv);
  e = add2(sub2(a, av), sub2(b, bv));
}

// (s, c) <- the renormalised pair of s + t, given |t| small against |s|
__device__ __forceinline__ void renorm2(float2 s, float2 t, DF2 &out) {
  float2 h = add2(s, t);
  out.c = sub2(t, sub2(h, s));
  out.s = h;
}

// acc += x * y componentwise, x = xh + xl, y = yh + yl
__device__ __forceinline__ void df_acc(DF2 &acc, float2 xh, float2 xl, float2 yh, float2 yl) {
  float2 p = __fmul2_rn(xh, yh);
  float2 e = __ffma2_rn(xh, yh, neg2(p));
  e = __ffma2_rn(xh, yl, e);
  e = __ffma2_rn(xl, yh, e);
  float2 s, t;
  two_sum2(acc.s, p, s, t);
  renorm2(s, add2(t, add2(acc.c, e)), acc);
}

// a += b
__device__ __forceinline__ void df_add(DF2 &a, DF2 b) {
  float2 s, t;
  two_sum2(a.s, b.s, s, t);
  renorm2(s, add2(t, add2(a.c, b.c)), a);
}

__device__ __forceinline__ float4 ld4(const zdf *p) { return *(const float4 *)p; }
__device__ __forceinline__ void st4(zdf *p, float2 h, float2 l) { *(float4 *)p = make_float4(h.x, h.y, l.x, l.y); }

#define KCH_DF 8  // dots per launch of k_mdot_df (registers: two running sums per dot)

// part[b][k][r][0..1] = this block's (A, B) sums for V_k^H w:
// A = sum (vr wr, vi wi), B = sum (vr wi, vi wr), so that
// Re = A.x + A.y and Im = B.x - B.y.  Same thread layout as k_mdot.
template <int KC>
__global__ void __launch_bounds__(256, 2) k_mdot_df(const zdf *__restrict__ V, long vstride,
                                                    const zdf *__restrict__ w, long E, int R,
                                                    float4 *__restrict__ part) {
  __shared__ float4 sm[2][256];
  int t = threadIdx.x, nt = blockDim.x;
  int G = nt / R, q = t / R;
  DF2 A[KC], B[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) A[k] = B[k] = DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  long stride = (long)gridDim.x * nt;
  for (long e = (long)blockIdx.x * nt + t; e < E; e += stride) {
    float4 wv = ld4(w + e);
    float2 wh = make_float2(wv.x, wv.y), wl = make_float2(wv.z, wv.w);
    float2 sh = swap2(wh), sl = swap2(wl);
    float4 v[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) v[k] = ld4(V + k * vstride + e);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      float2 vh = make_float2(v[k].x, v[k].y), vl = make_float2(v[k].z, v[k].w);
      df_acc(A[k], vh, vl, wh, wl);
      df_acc(B[k], vh, vl, sh, sl);
    }
  }
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    sm[0][t] = make_float4(A[k].s.x, A[k].s.y, A[k].c.x, A[k].c.y);
    sm[1][t] = make_float4(B[k].s.x, B[k].s.y, B[k].c.x, B[k].c.y);
    __syncthreads();
    for (int s = G >> 1; s > 0; s >>= 1) {
      if (q < s)
        for (int h = 0; h < 2; ++h) {
          float4 x = sm[h][t], y = sm[h][t + s * R];
          DF2 a{make_float2(x.x, x.y), make_float2(x.z, x.w)};
          df_add(a, DF2{make_float2(y.x, y.y), make_float2(y.z, y.w)});
          sm[h][t] = make_float4(a.s.x, a.s.y, a.c.x, a.c.y);
        }
      __syncthreads();
    }
    if (q == 0) {
      float4 *o = part + (((long)blockIdx.x * KC + k) * R + t) * 2;
      o[0] = sm[0][t];
      o[1] = sm[1][t];
    }
    __syncthreads();
  }
}

static void launch_mdot_df(int kc, int nblk, int nt, cudaStream_t s, const zdf *V, long vstride, const zdf *w,
                           long E, int R, float4 *part) {
  switch (kc) {
#define WL_MDOT_DF(K) \
  case K: k_mdot_df<K><<<nblk, nt, 0, s>>>(V, vstride, w, E, R, part); break;
    WL_MDOT_DF(1) WL_MDOT_DF(2) WL_MDOT_DF(3) WL_MDOT_DF(4) WL_MDOT_DF(5) WL_MDOT_DF(6) WL_MDOT_DF(7) WL_MDOT_DF(8)
#undef WL_MDOT_DF
    default: break;
  }
}

// a coefficient c as the two pre-broadcast double-float pairs k_maxpy_df and
// k_xupd_df read: {crh, crh, crl, crl} and {cih, -cih, cil, -cil}
__device__ __forceinline__ void put_coef_df(float4 *c, zd s) {
  float2 cr = split_df(s.re), cim = split_df(s.im);
  c[0] = make_float4(cr.x, cr.x, cr.y, cr.y);
  c[1] = make_float4(cim.x, -cim.x, cim.y, -cim.y);
}

// the sums of k_mdot_df over blocks, one warp per (k, r) in a fixed order,
// converted to FP64: out[r][k0 + k] (= or +=) V_k^H w; with coef, the
// coefficients for k_maxpy_df: {crh, crh, crl, crl} and {cih, -cih, cil, -cil}
__global__ void k_mdot_final_df(const float4 *__restrict__ part, int nblk, int kc, int R, zd *out, int ostride,
                                int k0, int accumulate, float4 *coef) {
  int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= kc * R) return;
  int k = wid / R, r = wid % R;
  DF2 A{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, B = A;
  for (int b = lane; b < nblk; b += 32) {
    const float4 *p = part + (((long)b * kc + k) * R + r) * 2;
    float4 x = p[0], y = p[1];
    df_add(A, DF2{make_float2(x.x, x.y), make_float2(x.z, x.w)});
    df_add(B, DF2{make_float2(y.x, y.y), make_float2(y.z, y.w)});
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    DF2 a2, b2;
    a2.s.x = __shfl_down_sync(0xffffffffu, A.s.x, off);
    a2.s.y = __shfl_down_sync(0xffffffffu, A.s.y, off);
    a2.c.x = __shfl_down_sync(0xffffffffu, A.c.x, off);
    a2.c.y = __shfl_down_sync(0xffffffffu, A.c.y, off);
    b2.s.x = __shfl_down_sync(0xffffffffu, B.s.x, off);
    b2.s.y = __shfl_down_sync(0xffffffffu, B.s.y, off);
    b2.c.x = __shfl_down_sync(0xffffffffu, B.c.x, off);
    b2.c.y = __shfl_down_sync(0xffffffffu, B.c.y, off);
    df_add(A, a2);
    df_add(B, b2);
  }
  if (lane) return;
  zd s = mk(((double)A.s.x + (double)A.s.y) + ((double)A.c.x + (double)A.c.y),
            ((double)B.s.x - (double)B.s.y) + ((double)B.c.x - (double)B.c.y));
  zd *o = out + (long)r * ostride + k0 + k;
  *o = accumulate ? (*o + s) : s;
  if (coef) put_coef_df(coef + ((long)(k0 + k) * R + r) * 2, s);
}

// w -= sum_k V_k c_k[r] in double-float (c from k_mdot_final_df): P sums
// (cr vr, cr vi) and Q sums (ci vr, -ci vi), so Re = P.x + Q.y and
// Im = P.y + Q.x; the k loop is unrolled by 4 with the loads issued first.
// With part != NULL the squared norm of the new w is summed as well, in the
// thread layout of k_mdot_df (a fixed grid, thread t on right-hand side
// t % R), and written as k_mdot_df's partials of one dot with B = 0: one
// pass over w instead of two.
__global__ void __launch_bounds__(256) k_maxpy_df(const zdf *__restrict__ V, long vstride, int kc,
                                                  const float4 *__restrict__ coef, zdf *__restrict__ w, long E,
                                                  int R, float4 *__restrict__ part) {
  __shared__ float4 sm[256];
  int t = threadIdx.x, nt = blockDim.x;
  DF2 N2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  long stride = (long)gridDim.x * nt;
  for (long e = (long)blockIdx.x * nt + t; e < E; e += stride) {
    int r = (int)(e % R);
    DF2 P{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, Q = P;
    auto step = [&](float4 v, float4 c0, float4 c1) {
      float2 vh = make_float2(v.x, v.y), vl = make_float2(v.z, v.w);
      df_acc(P, make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), vh, vl);
      df_acc(Q, make_float2(c1.x, c1.y), make_float2(c1.z, c1.w), vh, vl);
    };
    int k = 0;
    for (; k + 4 <= kc; k += 4) {
      float4 v[4], c[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = ld4(V + (k + u) * vstride + e);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 *cp = coef + ((long)(k + u) * R + r) * 2;
        c[u][0] = cp[0];
        c[u][1] = cp[1];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) step(v[u], c[u][0], c[u][1]);
    }
    for (; k < kc; ++k) {
      const float4 *cp = coef + ((long)k * R + r) * 2;
      step(ld4(V + k * vstride + e), cp[0], cp[1]);
    }
    df_add(P, DF2{swap2(Q.s), swap2(Q.c)});
    float4 wv = ld4(w + e);
    DF2 Wn{make_float2(wv.x, wv.y), make_float2(wv.z, wv.w)};
    df_add(Wn, DF2{neg2(P.s), neg2(P.c)});
    st4(w + e, Wn.s, Wn.c);
    if (part) df_acc(N2, Wn.s, Wn.c, Wn.s, Wn.c);
  }
  if (!part) return;
  int G = nt / R, q = t / R;
  sm[t] = make_float4(N2.s.x, N2.s.y, N2.c.x, N2.c.y);
  __syncthreads();
  for (int s = G >> 1; s > 0; s >>= 1) {
    if (q < s) {
      float4 x = sm[t], y = sm[t + s * R];
      DF2 a{make_float2(x.x, x.y), make_float2(x.z, x.w)};
      df_add(a, DF2{make_float2(y.x, y.y), make_float2(y.z, y.w)});
      sm[t] = make_float4(a.s.x, a.s.y, a.c.x, a.c.y);
    }
    __syncthreads();
  }
  if (q == 0) {
    float4 *o = part + ((long)blockIdx.x * R + t) * 2;
    o[0] = sm[t];
    o[1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// acc += x * y componentwise, x = xh + xl a double-float, y a float
__device__ __forceinline__ void df_acc1(DF2 &acc, float2 xh, float2 xl, float2 y) {
  float2 p = __fmul2_rn(xh, y);
  float2 e = __ffma2_rn(xh, y, neg2(p));
  e = __ffma2_rn(xl, y, e);
  float2 s, t;
  two_sum2(acc.s, p, s, t);
  renorm2(s, add2(t, add2(acc.c, e)), acc);
}

// the restart update x += sum_k Z_k y_k[r] (x FP64, Z the FP32 cycle
// outputs, y as pre-broadcast double-floats from k_trisolve): the sum in
// double-float, added to x in FP64 (the float parts widened exactly on the
// integer pipes)
__global__ void __launch_bounds__(256) k_xupd_df(const zf *__restrict__ Z, long zstride, int kc,
                                                 const float4 *__restrict__ coef, zd *__restrict__ x, long E, int R) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int r = (int)(e % R);
  DF2 P{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, Q = P;
  auto step = [&](zf z, float4 c0, float4 c1) {
    float2 zv = make_float2(z.re, z.im);
    df_acc1(P, make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), zv);
    df_acc1(Q, make_float2(c1.x, c1.y), make_float2(c1.z, c1.w), zv);
  };
  int k = 0;
  for (; k + 4 <= kc; k += 4) {
    zf v[4];
    float4 c[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = Z[(k + u) * zstride + e];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 *cp = coef + ((long)(k + u) * R + r) * 2;
      c[u][0] = cp[0];
      c[u][1] = cp[1];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) step(v[u], c[u][0], c[u][1]);
  }
  for (; k < kc; ++k) {
    const float4 *cp = coef + ((long)k * R + r) * 2;
    step(Z[k * zstride + e], cp[0], cp[1]);
  }
  df_add(P, DF2{swap2(Q.s), swap2(Q.c)});
  zd xv = x[e];
  xv.re += f2d(P.s.x) + f2d(P.c.x);
  xv.im += f2d(P.s.y) + f2d(P.c.y);
  x[e] = xv;
}

// v_{j+1} = f[rhs] w in double-float and its FP32 copy (the next cycle's
// input, the nearest float of hi + lo)
__global__ void k_scale_df(const zdf *__restrict__ in, zdf *__restrict__ out, zf *__restrict__ cyc,
                           const float2 *__restrict__ f, long E, int R) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  float2 fr = f[e % R];
  float2 ih = make_float2(fr.x, fr.x), il = make_float2(fr.y, fr.y);
  float4 wv = ld4(in + e);
  float2 wh = make_float2(wv.x, wv.y), wl = make_float2(wv.z, wv.w);
  float2 p = __fmul2_rn(wh, ih);
  float2 x = __ffma2_rn(wh, ih, neg2(p));
  x = __ffma2_rn(wh, il, x);
  x = __ffma2_rn(wl, ih, x);
  DF2 v;
  renorm2(p, x, v);
  st4(out + e, v.s, v.c);
  float2 c = add2(v.s, v.c);
  cyc[e] = mk(c.x, c.y);
}

// v_0 = f[rhs] r (r in FP64: the true residual) as a double-float, and its
// FP32 copy (the nearest float, as k_scale_rhs_cyc rounds)
__global__ void k_scale_first_df(const zd *__restrict__ in, zdf *__restrict__ out, zf *__restrict__ cyc,
                                 const double *__restrict__ f, long E, int R) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  zd v = f[e % R] * in[e];
  float2 re = split_df(v.re), im = split_df(v.im);
  st4(out + e, make_float2(re.x, im.x), make_float2(re.y, im.y));
  cyc[e] = mk(re.x, im.x);
}

// ------------------------------------------------------------------ Givens
// column j of the Arnoldi process for every active right-hand side
__global__ void k_givens(KS k, int j, double tol) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k.nrhs) return;
  int m = k.m;
  if (!k.active[r] || k.stop[r]) {
    k.inv[r] = 0.0;
    k.invdf[r] = make_float2(0.f, 0.f);
    return;
  }
  zd *hc = k.hcol + (long)r * (m + 1);
  double hn = sqrt(fmax(k.nrm2[r], 0.0));
  hc[j + 1] = mk(hn, 0.0);
  zd *cs = k.cs + (long)r * m;
  double *cc = k.cc + (long)r * m;
  for (int i = 0; i < j; ++i) {
    zd a = hc[i], b = hc[i + 1];
    zd t = cc[i] * a + cs[i] * b;
    hc[i + 1] = mk(0.0, 0.0) - cconj(cs[i]) * a + cc[i] * b;
    hc[i] = t;
  }
  double aa = sqrt(cnorm2(hc[j])), bb = hn;
  double den = sqrt(aa * aa + bb * bb);
  zd *g = k.g + (long)r * (m + 1);
  if (den == 0.0) {
    cc[j] = 1.0;
    cs[j] = mk(0.0, 0.0);
  } else if (aa == 0.0) {
    cc[j] = 0.0;
    cs[j] = mk(1.0, 0.0);
  } else {
    cc[j] = aa / den;
    zd ph = mk(hc[j].re / aa, hc[j].im / aa);
    cs[j] = (bb / den) * ph;  // conj(h_{j+1}) = h_{j+1} (real)
  }
  hc[j] = cc[j] * hc[j] + cs[j] * hc[j + 1];
  hc[j + 1] = mk(0.0, 0.0);
  zd gj = g[j];
  g[j + 1] = mk(0.0, 0.0) - cconj(cs[j]) * gj;
  g[j] = cc[j] * gj;
  zd *H = k.H + (long)r * (m + 1) * m;
  for (int i = 0; i <= j; ++i) H[i * m + j] = hc[i];
  k.iters[r] += 1;
  k.jend[r] = j + 1;
  double res = sqrt(cnorm2(g[j + 1]));
  bool bad = !isfinite(res);
  bool done = !(res > tol * k.bnorm[r]) || hn == 0.0 || bad;
  if (bad) {  // NaN / Inf seen: this right-hand side stops; the others go on
    k.running[1] = 1;
    k.nanf[r] = 1;
  }
  k.inv[r] = (done || hn == 0.0) ? 0.0 : 1.0 / hn;
  k.invdf[r] = split_df(k.inv[r]);
  if (done) k.stop[r] = 1;
  else atomicAdd(k.running, 1);
}

// y = H^-1 g (upper triangular, jend columns), zero beyond jend / inactive
// (with df, y also as double-float coefficients for k_xupd_df, in hpd)
__global__ void k_trisolve(KS k, int df) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k.nrhs) return;
  int m = k.m, je = k.active[r] ? k.jend[r] : 0;
  const zd *H = k.H + (long)r * (m + 1) * m;
  const zd *g = k.g + (long)r * (m + 1);
  zd *y = k.y + (long)r * m;
  for (int i = m - 1; i >= 0; --i) {
    if (i >= je) {
      y[i] = mk(0.0, 0.0);
      continue;
    }
    zd s = g[i];
    for (int q = i + 1; q < je; ++q) s = s - H[i * m + q] * y[q];
    zd d = H[i * m + i];
    double dn = cnorm2(d);
    y[i] = (dn > 0) ? mk((s.re * d.re + s.im * d.im) / dn, (s.im * d.re - s.re * d.im) / dn) : mk(0.0, 0.0);
  }
  for (int i = 0; i < m; ++i) k.yT[(long)i * k.nrhs + r] = y[i];
  if (df)
    for (int i = 0; i < m; ++i) put_coef_df(k.hpd + ((long)i * k.nrhs + r) * 2, y[i]);
}

// start of a cycle: beta = ||r||, inv = active ? 1/beta : 0, g = (beta, 0..)
__global__ void k_cycle_start(KS k) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k.nrhs) return;
  int m = k.m;
  double beta = sqrt(fmax(k.nrm2[r], 0.0));
  k.beta[r] = beta;
  bool act = k.active[r] && beta > 0.0;
  k.inv[r] = act ? 1.0 / beta : 0.0;
  k.invdf[r] = split_df(k.inv[r]);
  for (int i = 0; i <= m; ++i) k.g[(long)r * (m + 1) + i] = mk(0.0, 0.0);
  k.g[(long)r * (m + 1)] = mk(act ? beta : 0.0, 0.0);
  k.stop[r] = act ? 0 : 1;
  k.jend[r] = 0;
  for (int i = 0; i <= m; ++i) k.hcol[(long)r * (m + 1) + i] = mk(0.0, 0.0);
}

__global__ void k_zero_hcol(KS k) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k.nrhs) return;
  for (int i = 0; i <= k.m; ++i) k.hcol[(long)r * (k.m + 1) + i] = mk(0.0, 0.0);
}

// zero the entries (and squared norm) of the right-hand sides flagged in mask
__global__ void k_zero_masked(zd *__restrict__ v, long E, int R, const int *__restrict__ mask,
                              double *__restrict__ nrm2) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < E && mask[e % R]) v[e] = mk(0.0, 0.0);
  if (e < R && mask[e]) nrm2[e] = 0.0;
}

__global__ void k_re_of(const zd *a, double *b, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i].re;
}

namespace wl {

struct RedCfg {
  int R, nt, nblk;
};
static RedCfg red_cfg(long E, int R) {
  RedCfg c;
  c.R = R;
  int G = 1;
  while (R * G * 2 <= 256) G *= 2;
  c.nt = R * G;
  long want = (E + c.nt - 1) / c.nt;
  c.nblk = (int)std::max(1L, std::min(want, 608L));  // 4 blocks per SM on 152 SMs
  return c;
}

// out[r][k0+k] (=|+=) V_k^H w for k < kc, chunks of KCH
template <typename Tv>
static int mdots(wl_amg *a, const cx<Tv> *V, long vstride, int kc, const zd *w, long E, int R, zd *out,
                 int ostride, int accumulate, zd *copy_to, cudaStream_t s) {
  RedCfg c = red_cfg(E, R);
  // as few launches as possible, their dot counts as even as possible
  int nl = (kc + KCH - 1) / KCH;
  for (int k0 = 0, l = 0, kk = 0; k0 < kc; k0 += kk, ++l) {
    kk = (kc - k0 + (nl - l) - 1) / (nl - l);
    size_t sm = sizeof(zd) * kk * c.nt;
    wl_count_launches(2);
    launch_mdot<Tv>(kk, c.nblk, c.nt, sm, s, V + k0 * vstride, vstride, w, E, R, a->red.as<zd>());
    k_mdot_final<<<WL_GRID(kk * R * 32, 256), 256, 0, s>>>(a->red.as<zd>(), c.nblk, kk, R, out, ostride, k0,
                                                           accumulate, copy_to);
  }
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

// the same with double-float vectors; coef (or NULL) receives the
// coefficients for k_maxpy_df
static int mdots_df(wl_amg *a, const zdf *V, long vstride, int kc, const zdf *w, long E, int R, zd *out,
                    int ostride, int accumulate, float4 *coef, cudaStream_t s) {
  RedCfg c = red_cfg(E, R);
  int nl = (kc + KCH_DF - 1) / KCH_DF;
  for (int k0 = 0, l = 0, kk = 0; k0 < kc; k0 += kk, ++l) {
    kk = (kc - k0 + (nl - l) - 1) / (nl - l);
    wl_count_launches(2);
    launch_mdot_df(kk, c.nblk, c.nt, s, V + k0 * vstride, vstride, w, E, R, a->red.as<float4>());
    k_mdot_final_df<<<WL_GRID(kk * R * 32, 256), 256, 0, s>>>(a->red.as<float4>(), c.nblk, kk, R, out, ostride, k0,
                                                              accumulate, coef);
  }
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}


// w -= sum_k V_k coef_k and out[r] = |w_r|^2 in one pass (double-float)
static int maxpy_norm_df(wl_amg *a, const zdf *V, long vstride, int kc, const float4 *coef, zdf *w, long E, int R,
                         zd *tmp, double *out, cudaStream_t s) {
  RedCfg c = red_cfg(E, R);
  k_maxpy_df<<<c.nblk, c.nt, 0, s>>>(V, vstride, kc, coef, w, E, R, a->red.as<float4>());
  k_mdot_final_df<<<WL_GRID(R * 32, 256), 256, 0, s>>>(a->red.as<float4>(), c.nblk, 1, R, tmp, 1, 0, 0, nullptr);
  k_re_of<<<WL_GRID(R, 128), 128, 0, s>>>(tmp, out, R);
  wl_count_launches(3);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

static int norms2(wl_amg *a, const zd *w, long E, int R, zd *tmp, double *out, cudaStream_t s) {
  RedCfg c = red_cfg(E, R);
  k_norm2<<<c.nblk, c.nt, sizeof(double) * c.nt, s>>>(w, E, R, a->red.as<zd>());
  k_mdot_final<<<WL_GRID(R * 32, 256), 256, 0, s>>>(a->red.as<zd>(), c.nblk, 1, R, tmp, 1, 0, 0, nullptr);
  wl_count_launches(2);
  k_re_of<<<WL_GRID(R, 128), 128, 0, s>>>(tmp, out, R);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

// ||bh_r|| for every right-hand side (host output)
int fg_norms(wl_amg *a, const zd *v, int nrhs, double *out) {
  cudaStream_t s = a->op->stream;
  long E = (long)a->lev[0].n * 2 * nrhs;
  KS k = ks_layout(a->small.p, a->prm.fgmres_m, nrhs);
  zd *tmpc = a->small.as<zd>() + (a->small.bytes / sizeof(zd)) - 2 * (size_t)nrhs - 8;
  WL_TRY(norms2(a, v, E, nrhs, tmpc, k.nrm2, s));
  double *h_d = (double *)a->h_small;
  WL_CUDA(cudaMemcpyAsync(h_d, k.nrm2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  WL_CUDA(cudaStreamSynchronize(s));
  for (int r = 0; r < nrhs; ++r) out[r] = sqrt(h_d[r]);
  return WL_OK;
}

// true FP64 residual a->rr = bh - Dhat x and its norms (host output); the
// squared norms stay in the Krylov scalars for the next fg_cycle.  A
// right-hand side whose residual norm is not finite gets rnorm = NaN and its
// residual (and squared norm) zeroed, so no later kernel of the batch reads a
// non-finite value of it; the caller retires it with WL_NAN.
int fg_residual(wl_amg *a, const zd *bh, const zd *xh, int nrhs, double *rnorm) {
  wl_op *op = a->op;
  cudaStream_t s = op->stream;
  long E = (long)a->lev[0].n * 2 * nrhs;
  zd *w = a->w.as<zd>(), *rr = a->rr.as<zd>();
  WL_TRY(dhat_apply_dev(op, xh, 0, w, nrhs, s));
  k_sub<<<WL_GRID(E, 256), 256, 0, s>>>(bh, w, rr, E);
  wl_count_launches(1);
  KS k = ks_layout(a->small.p, a->prm.fgmres_m, nrhs);
  zd *tmpc = a->small.as<zd>() + (a->small.bytes / sizeof(zd)) - 2 * (size_t)nrhs - 8;
  WL_TRY(norms2(a, rr, E, nrhs, tmpc, k.nrm2, s));
  double *h_d = (double *)a->h_small;
  WL_CUDA(cudaMemcpyAsync(h_d, k.nrm2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  WL_CUDA(cudaStreamSynchronize(s));
  std::vector<int> bad(nrhs, 0);
  int nbad = 0;
  for (int r = 0; r < nrhs; ++r) {
    rnorm[r] = sqrt(h_d[r]);
    if (!std::isfinite(rnorm[r])) {
      rnorm[r] = NAN;
      bad[r] = 1;
      ++nbad;
    }
  }
  if (nbad) {
    WL_CUDA(cudaMemcpyAsync(k.nanf, bad.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
    k_zero_masked<<<WL_GRID(E, 256), 256, 0, s>>>(rr, E, nrhs, k.nanf, k.nrm2);
    wl_count_launches(1);
    WL_CUDA(cudaGetLastError());
    WL_CUDA(cudaStreamSynchronize(s));
  }
  return WL_OK;
}

// One restart cycle of FGMRES(m) from the residual left by fg_residual, for
// the right-hand sides with active[r] != 0 (the others are untouched):
// Arnoldi with z_j = M(v_j), Gram-Schmidt, Givens; then x += Z y.
// iters_out[r]: iterations this cycle ran for r (host); nan_out[r] (host, or
// NULL): 1 if r's Arnoldi residual became non-finite (r stopped there; its x
// is not to be trusted and the next true residual retires it).
int fg_cycle(wl_amg *a, const zd *bnorm_h, zd *xh, int nrhs, double tol, const int *active, int *iters_out,
             int *nan_out) {
  wl_op *op = a->op;
  cudaStream_t s = op->stream;
  int prec = a->prm.precision, m = a->prm.fgmres_m;
  long E = (long)a->lev[0].n * 2 * nrhs;
  long vs = E;
  KS k = ks_layout(a->small.p, m, nrhs);
  zd *V = a->V.as<zd>(), *w = a->w.as<zd>(), *rr = a->rr.as<zd>();
  zdf *Vd = a->V.as<zdf>(), *wd = a->w.as<zdf>();  // the same buffers with gs_arith = 1
  const bool df = a->prm.gs_arith == 1;
  size_t zb_ = prec_bytes(prec);
  char *Zb = (char *)a->Z.p;
  unsigned gE = WL_GRID(E, 256);
  double *h_d = (double *)a->h_small;
  (void)bnorm_h;
  WL_CUDA(cudaMemcpyAsync(k.active, active, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
  WL_CUDA(cudaMemsetAsync(k.iters, 0, sizeof(int) * nrhs, s));
  WL_CUDA(cudaMemsetAsync(k.nanf, 0, sizeof(int) * nrhs, s));
  // v_j = f[rhs] w is written together with the cycle-precision copy that
  // the cycle of step j reads (lev[0].f)
  auto scale_next = [&](const zd *in, zd *out) {
    if (prec == WL_FP64) k_scale_rhs_cyc<double><<<gE, 256, 0, s>>>(in, out, a->lev[0].f.as<zd>(), k.inv, E, nrhs);
    else k_scale_rhs_cyc<float><<<gE, 256, 0, s>>>(in, out, a->lev[0].f.as<zf>(), k.inv, E, nrhs);
    wl_count_launches(1);
  };
  k_cycle_start<<<WL_GRID(nrhs, 128), 128, 0, s>>>(k);
  wl_count_launches(1);
  if (df) {
    k_scale_first_df<<<gE, 256, 0, s>>>(rr, Vd, a->lev[0].f.as<zf>(), k.inv, E, nrhs);
    wl_count_launches(1);
  } else {
    scale_next(rr, V);
  }
  int jdone = 0;
  for (int j = 0; j < m; ++j) {
    void *zj = Zb + (size_t)j * vs * zb_;
    // z_j = M(v_j) in the cycle precision (lev[0].f holds v_j)
    WL_TRY(cycle_run(a, nrhs, prec, s));
    WL_CUDA(cudaMemcpyAsync(zj, a->lev[0].x.p, zb_ * E, cudaMemcpyDeviceToDevice, s));
    // w = Dhat z_j (FP64)
    if (df) WL_TRY(stencil_apply32_to_df(a, zj, wd, nrhs, s));
    else if (prec != WL_FP64 && a->prm.arnoldi_matvec == 1) WL_TRY(stencil_apply32_to64(a, zj, w, nrhs, s));
    else WL_TRY(dhat_apply_dev(op, zj, prec != WL_FP64, w, nrhs, s));
    // Gram-Schmidt against v_0 .. v_j
    k_zero_hcol<<<WL_GRID(nrhs, 128), 128, 0, s>>>(k);
    wl_count_launches(1);
    zd *tmpc = a->small.as<zd>() + (a->small.bytes / sizeof(zd)) - 2 * (size_t)nrhs - 8;
    for (int pass = 0; pass < a->prm.gs_passes; ++pass) {
      if (df) {
        WL_TRY(mdots_df(a, Vd, vs, j + 1, wd, E, nrhs, k.hcol, m + 1, 1, k.hpd, s));
        if (pass + 1 == a->prm.gs_passes) {  // the last pass also forms |w|^2
          WL_TRY(maxpy_norm_df(a, Vd, vs, j + 1, k.hpd, wd, E, nrhs, tmpc, k.nrm2, s));
        } else {
          k_maxpy_df<<<gE, 256, 0, s>>>(Vd, vs, j + 1, k.hpd, wd, E, nrhs, nullptr);
          wl_count_launches(1);
        }
      } else {
        WL_TRY(mdots<double>(a, V, vs, j + 1, w, E, nrhs, k.hcol, m + 1, 1, k.hpass, s));
        k_maxpy<double, 1><<<gE, 256, 0, s>>>(V, vs, j + 1, k.hpass, nrhs, w, E, nrhs);
        wl_count_launches(1);
      }
    }
    if (!df) WL_TRY(norms2(a, w, E, nrhs, tmpc, k.nrm2, s));
    WL_CUDA(cudaMemsetAsync(k.running, 0, sizeof(int) * 2, s));
    k_givens<<<WL_GRID(nrhs, 128), 128, 0, s>>>(k, j, tol);
    wl_count_launches(1);
    if (j + 1 < m) {
      if (df) {
        k_scale_df<<<gE, 256, 0, s>>>(wd, Vd + (j + 1) * vs, a->lev[0].f.as<zf>(), k.invdf, E, nrhs);
        wl_count_launches(1);
      } else {
        scale_next(w, V + (j + 1) * vs);
      }
    }
    WL_CUDA(cudaGetLastError());
    int run[2];
    WL_CUDA(cudaMemcpyAsync(h_d + nrhs, k.running, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    WL_CUDA(cudaStreamSynchronize(s));
    memcpy(run, h_d + nrhs, sizeof(int) * 2);
    jdone = j + 1;
    if (run[0] == 0) break;
  }
  k_trisolve<<<WL_GRID(nrhs, 128), 128, 0, s>>>(k, df ? 1 : 0);
  if (df) k_xupd_df<<<gE, 256, 0, s>>>(a->Z.as<zf>(), vs, jdone, k.hpd, xh, E, nrhs);
  else if (prec == WL_FP64) k_maxpy<double, 0><<<gE, 256, 0, s>>>(a->Z.as<zd>(), vs, jdone, k.yT, nrhs, xh, E, nrhs);
  else k_maxpy<float, 0><<<gE, 256, 0, s>>>(a->Z.as<zf>(), vs, jdone, k.yT, nrhs, xh, E, nrhs);
  wl_count_launches(2);
  WL_CUDA(cudaGetLastError());
  WL_CUDA(cudaMemcpyAsync(iters_out, k.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  if (nan_out) WL_CUDA(cudaMemcpyAsync(nan_out, k.nanf, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

// ||bhat|| per right-hand side for the stopping test inside fg_cycle
int fg_upload_bnorm(wl_amg *a, const double *bn, int nrhs) {
  KS k = ks_layout(a->small.p, a->prm.fgmres_m, nrhs);
  WL_CUDA(cudaMemcpyAsync(k.bnorm, bn, sizeof(double) * nrhs, cudaMemcpyHostToDevice, a->op->stream));
  WL_CUDA(cudaStreamSynchronize(a->op->stream));
  return WL_OK;
}

// restarted FGMRES on a fixed batch: every right-hand side runs until its
// true residual is <= tol * ||bhat|| or max_restarts cycles are spent; one
// whose residual becomes non-finite is retired with WL_NAN while the others
// go on.  Returns WL_NAN if any right-hand side was retired that way, else
// WL_NOT_CONVERGED if any missed tol, else WL_OK.
int fgmres_run(wl_amg *a, const zd *bh, zd *xh, int nrhs, double tol, wl_info *info) {
  std::vector<int> active(nrhs, 1), iters(nrhs, 0), restarts(nrhs, 0), it(nrhs, 0), nanr(nrhs, 0),
      nanc(nrhs, 0);
  std::vector<double> relres(nrhs, 0.0), bnorm(nrhs, 0.0), rn(nrhs, 0.0);
  WL_TRY(fg_norms(a, bh, nrhs, bnorm.data()));
  for (int r = 0; r < nrhs; ++r)
    if (!(bnorm[r] > 0)) bnorm[r] = 1.0;
  WL_TRY(fg_upload_bnorm(a, bnorm.data(), nrhs));
  int status = WL_OK;
  for (int cyc = 0;; ++cyc) {
    WL_TRY(fg_residual(a, bh, xh, nrhs, rn.data()));
    int any = 0;
    for (int r = 0; r < nrhs; ++r) {
      if (!std::isfinite(rn[r])) nanr[r] = 1;
      if (nanr[r]) {
        relres[r] = NAN;
        active[r] = 0;
        continue;
      }
      relres[r] = rn[r] / bnorm[r];
      active[r] = active[r] && relres[r] > tol && cyc < a->prm.max_restarts;
      any |= active[r];
    }
    if (!any) break;
    WL_TRY(fg_cycle(a, nullptr, xh, nrhs, tol, active.data(), it.data(), nanc.data()));
    for (int r = 0; r < nrhs; ++r) {
      iters[r] += it[r];
      if (active[r]) restarts[r]++;
    }
  }
  int nnan = 0;
  for (int r = 0; r < nrhs; ++r) {
    bool ok = !nanr[r] && relres[r] <= tol;
    if (nanr[r]) ++nnan;
    else if (!ok) status = WL_NOT_CONVERGED;
    if (info) {
      info[r].status = nanr[r] ? WL_NAN : ok ? WL_OK : WL_NOT_CONVERGED;
      info[r].restarts = restarts[r];
      info[r].iters = iters[r];
      info[r].true_relres = relres[r];
    }
  }
  if (nnan) {
    wl_set_error("non-finite residual for %d of %d right-hand sides", nnan, nrhs);
    return WL_NAN;
  }
  return status;
}

}  // namespace wl

#define MAX_BATCH 256

extern "C" int amg_fgmres(wl_amg *a, const void *bhat, void *x, int nrhs, double tol, wl_info *info) {
  if (!a || !bhat || !x || nrhs < 1 || nrhs > MAX_BATCH || !(tol > 0)) {
    wl_set_error("amg_fgmres: invalid argument (1 <= nrhs <= %d, tol > 0)", MAX_BATCH);
    return WL_EINVAL;
  }
  WL_TRY(wl::enter(a->op));
  WL_TRY(wl::ensure_workspace(a, nrhs, a->prm.precision));
  cudaStream_t s = a->op->stream;
  int n2 = a->lev[0].n * 2;
  WL_TRY(wl::to_internal((const zd *)bhat, a->bh.p, n2, nrhs, WL_FP64, s));
  WL_TRY(wl::to_internal((const zd *)x, a->xh.p, n2, nrhs, WL_FP64, s));
  int rc = wl::fgmres_run(a, a->bh.as<zd>(), a->xh.as<zd>(), nrhs, tol, info);
  if (rc < 0 && rc != WL_NAN) return rc;
  WL_TRY(wl::from_internal(a->xh.p, (zd *)x, n2, nrhs, WL_FP64, s));
  WL_CUDA(cudaStreamSynchronize(s));
  if (wl::tile_timeout_take(s)) return WL_TIMEOUT;
  return rc;
}

// e -= z, z in the cycle precision (widened exactly to double)
template <typename Tz>
__global__ void k_sub_inplace(zd *__restrict__ e, const cx<Tz> *__restrict__ z, long E) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E) {
    zd w = widen<double>(z[i]);
    e[i].re -= w.re;
    e[i].im -= w.im;
  }
}

// Sec. 4's convergence estimate: the configured cycle as a stationary
// iteration on Dhat x = 0, e <- e - M(Dhat e), Dhat in FP64, M in the
// hierarchy's precision; per right-hand side rho = |e^nu| / |e^(nu-1)| at
// the first nu with |e^nu| <= tol |e^0| or at nu = maxit.
extern "C" int amg_rho(wl_amg *a, const void *x0, void *x, int nrhs, double tol, int maxit, double *rho,
                       int *iters, double *hist) {
  if (!a || !x0 || !x || !rho || !iters || nrhs < 1 || nrhs > MAX_BATCH || !(tol >= 0) || maxit < 1) {
    wl_set_error("amg_rho: invalid argument (1 <= nrhs <= %d, tol >= 0, maxit >= 1)", MAX_BATCH);
    return WL_EINVAL;
  }
  int prec = a->prm.precision;
  WL_TRY(wl::enter(a->op));
  WL_TRY(wl::ensure_workspace(a, nrhs, prec));
  cudaStream_t s = a->op->stream;
  int n2 = a->lev[0].n * 2;
  long E = (long)n2 * nrhs;
  unsigned gE = WL_GRID(E, 256);
  zd *e = a->xh.as<zd>(), *w = a->w.as<zd>();
  WL_TRY(wl::to_internal((const zd *)x0, e, n2, nrhs, WL_FP64, s));
  std::vector<double> n0(nrhs), prev(nrhs), cur(nrhs);
  std::vector<int> done(nrhs, 0);
  WL_TRY(wl::fg_norms(a, e, nrhs, n0.data()));
  for (int r = 0; r < nrhs; ++r) {
    prev[r] = n0[r];
    rho[r] = 0;
    iters[r] = 0;
    if (hist) hist[(size_t)r * (maxit + 1)] = n0[r];
  }
  int left = nrhs, diverged = 0;
  for (int nu = 1; nu <= maxit && left > 0; ++nu) {
    WL_TRY(wl::dhat_apply_dev(a->op, e, 0, w, nrhs, s));
    if (prec == WL_FP64) {
      WL_CUDA(cudaMemcpyAsync(a->lev[0].f.p, w, sizeof(zd) * E, cudaMemcpyDeviceToDevice, s));
    } else {
      k_cast<float, double><<<gE, 256, 0, s>>>(w, a->lev[0].f.as<zf>(), E);
      wl_count_launches(1);
    }
    WL_TRY(wl::cycle_run(a, nrhs, prec, s));
    if (prec == WL_FP64) k_sub_inplace<double><<<gE, 256, 0, s>>>(e, a->lev[0].x.as<zd>(), E);
    else k_sub_inplace<float><<<gE, 256, 0, s>>>(e, a->lev[0].x.as<zf>(), E);
    wl_count_launches(1);
    WL_CUDA(cudaGetLastError());
    WL_TRY(wl::fg_norms(a, e, nrhs, cur.data()));
    for (int r = 0; r < nrhs; ++r) {
      if (done[r]) continue;
      if (!std::isfinite(cur[r])) {  // diverged past overflow: keep the last finite ratio
        done[r] = 1;
        --left;
        ++diverged;
        continue;
      }
      rho[r] = prev[r] > 0 ? cur[r] / prev[r] : 0;
      iters[r] = nu;
      if (hist) hist[(size_t)r * (maxit + 1) + nu] = cur[r];
      prev[r] = cur[r];
      if (cur[r] <= tol * n0[r]) {
        done[r] = 1;
        --left;
      }
    }
  }
  WL_TRY(wl::from_internal(e, (zd *)x, n2, nrhs, WL_FP64, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return (left || diverged) ? WL_NOT_CONVERGED : WL_OK;
}

// reduce, FGMRES, reconstruct for n right-hand sides on the lane L (its own
// stream and workspace); returns the fgmres_run status or an error
static int solve_lane(wl_amg *L, const zd *bb, zd *xx, int n, double tol, wl_info *info) {
  wl_op *op = L->op;
  cudaStream_t s = op->stream;
  WL_TRY(wl::ensure_workspace(L, n, L->prm.precision));
  WL_TRY(wl::eo_reduce_internal(op, bb, L->bh.as<zd>(), n, s));
  if (L->prm.zero_guess)
    WL_CUDA(cudaMemsetAsync(L->xh.p, 0, sizeof(zd) * (size_t)L->lev[0].n * 2 * n, s));
  else
    WL_TRY(wl::take_even_internal(op, xx, L->xh.as<zd>(), n, s));
  int rc = wl::fgmres_run(L, L->bh.as<zd>(), L->xh.as<zd>(), n, tol, info);
  if (rc < 0 && rc != WL_NAN) return rc;
  WL_TRY(wl::eo_reconstruct_internal(op, bb, L->xh.as<zd>(), xx, n, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return rc;
}

static int combine(int a, int b) {
  if (a == WL_NAN || b == WL_NAN) return WL_NAN;
  return (a || b) ? WL_NOT_CONVERGED : WL_OK;
}

// the host-buffer form of solve_lane: b (and x, unless zero_guess) copied to
// the device staging db / dx on the lane's stream, solved there, x copied
// back on the same stream, so one lane's copies overlap the other lane's
// solve
static int solve_lane_host(wl_amg *L, const zd *hb, zd *hx, zd *db, zd *dx, int n, double tol, wl_info *info) {
  cudaStream_t s = L->op->stream;
  size_t bytes = sizeof(zd) * (size_t)L->op->N * L->op->N * 2 * n;
  WL_CUDA(cudaMemcpyAsync(db, hb, bytes, cudaMemcpyHostToDevice, s));
  if (!L->prm.zero_guess) WL_CUDA(cudaMemcpyAsync(dx, hx, bytes, cudaMemcpyHostToDevice, s));
  int rc = solve_lane(L, db, dx, n, tol, info);
  if (rc < 0 && rc != WL_NAN) return rc;
  WL_CUDA(cudaMemcpyAsync(hx, dx, bytes, cudaMemcpyDeviceToHost, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return rc;
}

// two halves of the batch at the same time: lane(L, r0, n, info) for the
// first half on a's stream in this thread, for the second on the twin's
// stream in a second host thread (both drive their own FGMRES, with their
// own host synchronisations), so one half's Gram-Schmidt kernels can share
// the GPU with the other half's cycle
template <class Lane>
static int run_two_lanes(wl_amg *a, int nb, wl_info *info, Lane lane) {
  if (!a->twin) {
    a->twin = wl::make_twin(a);
    if (!a->twin) return WL_ECUDA;
  }
  wl_amg *t = a->twin;
  int keep_cap = t->cap;
  t->prm = a->prm;
  t->prm.overlap = 0;
  t->cap = keep_cap;
  const int h0 = (nb + 1) / 2, h1 = nb - h0, prec = a->prm.precision;
  // Workspaces, launch forms and cycle graphs of both lanes are made here,
  // before the second thread starts, so that neither lane times kernels or
  // captures a graph while the other one runs.  The twin takes a's launch
  // forms for its width (measured on a, or pinned there) unless it already
  // holds a graph of that width.
  WL_TRY(wl::ensure_workspace(a, h0, prec));
  WL_TRY(wl::cycle_prepare(a, h0, prec, a->op->stream, nullptr));
  if (h1 != h0) WL_TRY(wl::autotune_sweeps(a, h1, prec, a->op->stream));
  bool t_has_graph = false;
  for (const auto &g : t->graphs) t_has_graph |= (g.nrhs == h1 && g.prec == prec);
  if (!t_has_graph)
    for (int l = 0; l < a->L; ++l) {
      std::vector<KTune> &tv = t->lev[l].tune;
      for (const KTune &k : a->lev[l].tune) {
        if (k.nrhs != h1 || k.prec != prec) continue;
        bool set = false;
        for (KTune &q : tv)
          if (q.nrhs == h1 && q.prec == prec && (q.form == 2) == (k.form == 2)) {
            q = k;
            set = true;
          }
        if (!set) tv.push_back(k);
      }
    }
  WL_TRY(wl::enter(t->op));  // the twin's stream waits for a's (which waits for the caller's)
  WL_TRY(wl::ensure_workspace(t, h1, prec));
  WL_TRY(wl::cycle_prepare(t, h1, prec, t->op->stream, nullptr));
  int rc1 = WL_OK;
  std::string err1;
  std::thread th([&] {
    if (cudaSetDevice(t->op->device) != cudaSuccess) {
      rc1 = WL_ECUDA;
      err1 = "second solve lane: cudaSetDevice failed";
      return;
    }
    rc1 = lane(t, h0, h1, info ? info + h0 : nullptr);
    if (rc1 < 0 && rc1 != WL_NAN) err1 = wl_last_error();
  });
  int rc0 = lane(a, 0, h0, info);
  th.join();
  if (rc1 < 0 && rc1 != WL_NAN) {
    wl_set_error("%s", err1.c_str());
    return rc1;
  }
  if (rc0 < 0 && rc0 != WL_NAN) return rc0;
  if (rc0 == WL_NAN || rc1 == WL_NAN)
    wl_set_error("non-finite residual for some right-hand sides");
  return combine(rc0, rc1);
}

static int solve_two_lanes(wl_amg *a, const zd *bb, zd *xx, int nb, double tol, wl_info *info) {
  const size_t fs = (size_t)a->op->N * a->op->N * 2;
  return run_two_lanes(a, nb, info, [&](wl_amg *L, int r0, int n, wl_info *inf) {
    return solve_lane(L, bb + r0 * fs, xx + r0 * fs, n, tol, inf);
  });
}

extern "C" int amg_solve(wl_amg *a, const void *b, void *x, int nrhs, double tol, wl_info *info) {
  if (!a || !b || !x || nrhs < 1 || !(tol > 0)) {
    wl_set_error("amg_solve: invalid argument");
    return WL_EINVAL;
  }
  wl_op *op = a->op;
  WL_TRY(wl::enter(op));
  cudaStream_t s = op->stream;
  int N = op->N;
  int status = WL_OK;
  for (int r0 = 0; r0 < nrhs; r0 += MAX_BATCH) {
    int nb = std::min(MAX_BATCH, nrhs - r0);
    const zd *bb = (const zd *)b + (size_t)r0 * N * N * 2;
    zd *xx = (zd *)x + (size_t)r0 * N * N * 2;
    int rc = (a->prm.overlap && nb >= 32) ? solve_two_lanes(a, bb, xx, nb, tol, info ? info + r0 : nullptr)
                                          : solve_lane(a, bb, xx, nb, tol, info ? info + r0 : nullptr);
    if (rc < 0 && rc != WL_NAN) return rc;
    status = combine(status, rc);
  }
  WL_CUDA(cudaStreamSynchronize(s));
  if (wl::tile_timeout_take(s)) return WL_TIMEOUT;
  return status;
}

extern "C" int amg_solve_host(wl_amg *a, const void *b, void *x, int nrhs, double tol, wl_info *info) {
  if (!a || !b || !x || nrhs < 1 || !(tol > 0)) {
    wl_set_error("amg_solve_host: invalid argument");
    return WL_EINVAL;
  }
  wl_op *op = a->op;
  WL_TRY(wl::enter(op));
  cudaStream_t s = op->stream;
  const size_t fs = (size_t)op->N * op->N * 2;
  const int nbmax = std::min(MAX_BATCH, nrhs);
  WL_TRY(a->sb.alloc(sizeof(zd) * fs * nbmax));
  WL_TRY(a->sx.alloc(sizeof(zd) * fs * nbmax));
  zd *db = a->sb.as<zd>(), *dx = a->sx.as<zd>();
  int status = WL_OK;
  for (int r0 = 0; r0 < nrhs; r0 += MAX_BATCH) {
    int nb = std::min(MAX_BATCH, nrhs - r0);
    const zd *hb = (const zd *)b + (size_t)r0 * fs;
    zd *hx = (zd *)x + (size_t)r0 * fs;
    auto lane = [&](wl_amg *L, int q0, int n, wl_info *inf) {
      return solve_lane_host(L, hb + q0 * fs, hx + q0 * fs, db + q0 * fs, dx + q0 * fs, n, tol, inf);
    };
    wl_info *ib = info ? info + r0 : nullptr;
    int rc = (a->prm.overlap && nb >= 32) ? run_two_lanes(a, nb, ib, lane) : lane(a, 0, nb, ib);
    if (rc < 0 && rc != WL_NAN) return rc;
    status = combine(status, rc);
  }
  WL_CUDA(cudaStreamSynchronize(s));
  if (wl::tile_timeout_take(s)) return WL_TIMEOUT;
  return status;
}

// ------------------------------------------------------------ instrumentation
// FP64 FMA throughput probe: FMA_CHAINS independent chains of FMA_STEPS
// dependent FMAs per thread (v <- v b + c with 0 < b < 1, so every value
// stays finite); the one conditional store keeps the chains live.
constexpr int FMA_CHAINS = 8, FMA_STEPS = 4096, FMA_BLOCKS_PER_SM = 8;
__global__ void __launch_bounds__(256) k_fp64_fma(double *out, double b, double c) {
  double v[FMA_CHAINS];
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; ++i) v[i] = 1e-3 * threadIdx.x + i;
  for (int it = 0; it < FMA_STEPS; ++it)
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) v[i] = fma(v[i], b, c);
  double s = 0;
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; ++i) s += v[i];
  if (s == 0.0) out[0] = s;
}

extern "C" int wl_time_kernel(wl_amg *a, int kind, int level, int nrhs, int prec, int reps, double *avg_ms) {
  if (!a || !avg_ms || nrhs < 1 || nrhs > MAX_BATCH || reps < 1 || level < 0 || level >= a->L ||
      (prec != WL_FP64 && prec != WL_FP32 && prec != WL_FP32_BF16) || kind < WL_K_DHAT || kind > WL_K_FP64_FMA ||
      ((kind == WL_K_KACZ || kind == WL_K_STENCIL || kind == WL_K_RESTRICT || kind == WL_K_PROLONG ||
        kind == WL_K_KACZ_TILE) &&
       level == a->L - 1)) {
    wl_set_error("wl_time_kernel: invalid argument");
    return WL_EINVAL;
  }
  WL_TRY(wl::enter(a->op));
  WL_TRY(wl::ensure_workspace(a, nrhs, prec));
  cudaStream_t s = a->op->stream;
  int m = a->prm.fgmres_m;
  long E = (long)a->lev[0].n * 2 * nrhs;
  int kc = std::min(11, m + 1);
  KS k = ks_layout(a->small.p, m, nrhs);
  Level &L = a->lev[level];
  auto launch = [&](int rep) -> int {
    switch (kind) {
      case WL_K_DHAT: return wl::dhat_apply_dev(a->op, a->Z.p, prec != WL_FP64, a->w.as<zd>(), nrhs, s);
      case WL_K_KACZ: return wl::kaczmarz_colour(a, level, prec, L.x.p, L.r.p, nrhs, rep & 15, s);
      case WL_K_KACZ_TILE: {  // the autotuned form where the level has one, else the default chunk
        KTune t = wl::sweep_form_of(a, level, prec, nrhs);
        return wl::kaczmarz_tile(a, level, prec, L.x.p, L.r.p, nrhs, rep & 3, s, t.form == 2 ? t.param : 0);
      }
      case WL_K_STENCIL: return wl::stencil_apply(a, level, prec, L.x.p, L.r.p, L.f.p, nrhs, s);
      case WL_K_RESTRICT: return wl::restrict_op(a, level, prec, L.r.p, a->lev[level + 1].f.p, nrhs, s);
      case WL_K_PROLONG: return wl::prolong_op(a, level, prec, a->lev[level + 1].x.p, L.x.p, nrhs, s);
      case WL_K_COARSEST:
        return wl::coarsest_apply(a, prec, a->lev[a->L - 1].f.p, a->lev[a->L - 1].x.p, nrhs, s);
      case WL_K_GS_DOT:  // the Gram-Schmidt arithmetic the hierarchy's solves use
        if (a->prm.gs_arith == 1)
          return wl::mdots_df(a, a->V.as<zdf>(), E, kc, a->w.as<zdf>(), E, nrhs, k.hcol, m + 1, 0, k.hpd, s);
        return wl::mdots<double>(a, a->V.as<zd>(), E, kc, a->w.as<zd>(), E, nrhs, k.hcol, m + 1, 0, k.hpass, s);
      case WL_K_FP64_FMA: {
        int nsm = 0;
        WL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, a->op->device));
        k_fp64_fma<<<nsm * FMA_BLOCKS_PER_SM, 256, 0, s>>>((double *)a->w.p, 0.999, 1e-3);
        wl_count_launches(1);
        return WL_OK;
      }
      default:
        if (a->prm.gs_arith == 1)
          k_maxpy_df<<<WL_GRID(E, 256), 256, 0, s>>>(a->V.as<zdf>(), E, kc, k.hpd, a->w.as<zdf>(), E, nrhs, nullptr);
        else
          k_maxpy<double, 1><<<WL_GRID(E, 256), 256, 0, s>>>(a->V.as<zd>(), E, kc, k.hpass, nrhs, a->w.as<zd>(), E,
                                                              nrhs);
        wl_count_launches(1);
        return WL_OK;
    }
  };
  WL_TRY(launch(0));
  cudaEvent_t e0, e1;
  WL_CUDA(cudaEventCreate(&e0));
  WL_CUDA(cudaEventCreate(&e1));
  int rc = WL_OK;
  if (cudaEventRecord(e0, s) != cudaSuccess) rc = WL_ECUDA;
  for (int i = 0; i < reps && !rc; ++i) rc = launch(i + 1);
  float ms = 0;
  if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = WL_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  WL_CUDA(cudaGetLastError());
  *avg_ms = (double)ms / reps;
  return WL_OK;
}
