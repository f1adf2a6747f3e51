// wl_agg.cu -- aggregation coarse space on the GPU: the interpolation P and
// the Galerkin operator P^H A P, and the coarse block-stencil apply on CUDA
// cores and on the tensor cores (tcgen05).
//
// Sec. 4 closes by naming the alternative to its W-cycles that it did not
// explore: more interpolation variables per coarse point.  Here every B x B
// cell of the full coarsening (Sec. 3.2) is an aggregate; for each aggregate
// and spin the k test vectors restricted there are orthonormalised (modified
// Gram-Schmidt, in their given order), and those columns are P's columns, so
// a coarse site carries 2k variables (k per spin; Gamma5 P = P Gamma5c) and
// the Galerkin operator of Sec. 3.5 is a 9-point stencil of dense 2k x 2k
// complex blocks.  Its apply, y_h = sum_d A[h][d] x_{neighbour(h, d)}, is for
// many right-hand sides a batch of small dense complex products: the place
// where tensor cores pay.
//
// Layouts.  Q [nc][2][B*B][k] (coarse site, spin, member ia B + ib, column),
// Ac [nc][9][2k][2k] (row = 2k variable of h, column = variable of the
// neighbour), complex128 masters; the apply runs on FP32 copies with the
// internal vector layout [nc][nrhs][2k] (site, right-hand side, variable).
//
// Tensor-core apply (k = 8, 2k = 16).  Per coarse site and chunk of 64
// right-hand sides, one accumulation D (128 x 16, FP32, in tensor memory):
// row 2r + p of D holds p = 0: Re y_r, p = 1: Im y_r, column c the variable.
// With K running over (offset d, variable j, re/im u):
//   A[2r+0][(d,j,0)] = Re x, A[2r+0][(d,j,1)] = -Im x,
//   A[2r+1][(d,j,0)] = Im x, A[2r+1][(d,j,1)] =  Re x   (x = x_r of neighbour d, variable j)
//   B[(d,j,0)][c]    = Re Ac[h][d][c][j], B[(d,j,1)][c] = Im Ac[h][d][c][j],
// so D[2r][c] = sum Re(a) Re(x) - Im(a) Im(x) = Re(a x) and D[2r+1][c] =
// Im(a x).  B is the stencil block itself read K-major (row c is the 16
// complex coefficients, re/im interleaved); A is built from x by the threads
// and written straight into tensor memory (tcgen05.st), so only B passes
// through shared memory.  FP32 accuracy from TF32 operands: every operand is
// split v = hi + lo with hi, lo TF32 (round to nearest), and the result is
// hi*hi + hi*lo + lo*hi (the dropped lo*lo is below 2^-22 relative).  The
// tensor cores add the products of one MMA to the accumulator with
// truncation, so a long chain of MMAs into one accumulator drifts (measured:
// 2.5e-6 relative over the 108 MMAs of a site).  The hi*hi products are
// therefore spread over three accumulators (offsets d = 0-2, 3-5, 6-8: 12
// MMAs each), the two correction terms go to a fourth, and the epilogue adds
// the four in FP32 (round to nearest).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "wl_common.cuh"

struct wl_agg {
  wl_amg *amg;  // hierarchy whose level `level` is the fine side (retained)
  int level, B, k, M, Nf, Nc, nf, nc;
  Geo gf, gc;
  DBuf Q, Ac, Ac32;  // complex128 masters, FP32 copy of Ac
  DBuf X, Y;         // internal FP32 vectors [nc][nrhs][2k], `cap` right-hand sides
  DBuf X64, Y64;     // internal FP64 vectors for the FP64 apply
  int cap, cap64;
  DBuf flag;         // device status word (rank deficiency, tensor-core wait timeout)
};

// ------------------------------------------------------------- geometry
// fine site of member m = ia B + ib of coarse site hc: the cell corner of hc
// is the fine point (xc B, yc B), i.e. (a0, b0) = ((xc + yc) B / 2, (xc - yc) B / 2)
__device__ __forceinline__ int agg_fine_site(const Geo &gf, const Geo &gc, int B, int hc, int m) {
  int xc, yc;
  gc.xy(hc, xc, yc);
  int a0 = (xc + yc) * B / 2, b0 = (xc - yc) * B / 2;
  int a = a0 + m / B, b = b0 + m % B;
  return gf.idx(a + b, a - b);
}

__device__ __forceinline__ int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// coarse site and member index of fine site h
__device__ __forceinline__ void agg_member(const Geo &gf, const Geo &gc, int B, int h, int &hc, int &m) {
  int x, y;
  gf.xy(h, x, y);
  int a = (x + y) >> 1, b = (x - y) / 2;
  int a0 = B * fdiv(a, B), b0 = B * fdiv(b, B);
  int xf = (a0 + b0) & (gf.N - 1), yf = (a0 - b0) & (gf.N - 1);
  hc = gc.idx(xf / B, yf / B);
  m = (a - a0) * B + (b - b0);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------- interpolation P
// one warp per (coarse site, spin); lane m < B*B holds member m; the k
// columns sit in shared memory, [warp][m][k]
__global__ void k_agg_interp(Geo gf, Geo gc, int B, int k, const zd *__restrict__ V, long vstride,
                             zd *__restrict__ Q, int *flag) {
  extern __shared__ zd qs_all[];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, M = B * B;
  long task = (long)blockIdx.x * (blockDim.x >> 5) + warp;
  if (task >= 2L * gc.nsites()) return;  // whole warps leave together
  int hc = (int)(task >> 1), s = (int)(task & 1);
  zd *q = qs_all + (long)warp * 32 * k;
  bool mine = lane < M;
  if (mine) {
    int h = agg_fine_site(gf, gc, B, hc, lane);
    for (int kap = 0; kap < k; ++kap) q[lane * k + kap] = V[kap * vstride + 2 * (long)h + s];
  }
  for (int kap = 0; kap < k; ++kap) {
    zd v = mine ? q[lane * k + kap] : mk(0.0, 0.0);
    double n0 = warp_sum(cnorm2(v));
    for (int lam = 0; lam < kap; ++lam) {
      zd u = mine ? q[lane * k + lam] : mk(0.0, 0.0);
      zd t = cmulc(u, v);  // conj(q_lambda) q_kappa
      zd dt = mk(warp_sum(t.re), warp_sum(t.im));
      v = v - dt * u;
    }
    double nn = warp_sum(cnorm2(v));
    if (!(sqrt(nn) > 1e-12 * sqrt(n0))) {
      if (lane == 0) atomicExch(flag, 1);
      nn = 1.0;
    }
    double nr = sqrt(nn);
    v = mk(v.re / nr, v.im / nr);
    if (mine) q[lane * k + kap] = v;
  }
  if (mine)
    for (int kap = 0; kap < k; ++kap) Q[(((long)hc * 2 + s) * M + lane) * k + kap] = q[lane * k + kap];
}

// --------------------------------------------------------------- Galerkin
// one block per coarse site hc: Ac[hc][dc][(s,kappa)][(t,lambda)] =
// sum over members i of hc and fine offsets d' whose neighbour j lies in the
// coarse neighbour dc of conj(Q_i[s][kappa]) A_l[i][d'][s][t] Q_j[t][lambda]
// (members ascending, then d' ascending).  Shared memory: Q of the nine
// coarse neighbours [9][2][M][k], the members' stencil rows [M][9][2][2] and
// the (dc, member of j) table [M][9].
__global__ void k_agg_galerkin(Geo gf, Geo gc, int B, int k, const zd *__restrict__ A, const zd *__restrict__ Q,
                               zd *__restrict__ Ac) {
  extern __shared__ zd gs_all[];
  int M = B * B, K2 = 2 * k, hc = blockIdx.x, tid = threadIdx.x;
  zd *Qs = gs_all;                       // [9][2][M][k]
  zd *As = Qs + 9 * 2 * M * k;           // [M][36]
  int *tab = (int *)(As + M * 36);       // [M][9]: (dc << 8) | member of j, or -1
  int xc, yc;
  gc.xy(hc, xc, yc);
  for (int e = tid; e < 9 * 2 * M * k; e += blockDim.x) {
    int dc = e / (2 * M * k), rest = e % (2 * M * k);
    Qs[e] = Q[(long)gc.nb(xc, yc, dc) * 2 * M * k + rest];
  }
  for (int e = tid; e < M * 36; e += blockDim.x) {
    int i = e / 36;
    As[e] = A[(long)agg_fine_site(gf, gc, B, hc, i) * 36 + e % 36];
  }
  for (int e = tid; e < M * 9; e += blockDim.x) {
    int i = e / 9, d = e % 9, x, y, hj, mj, dc = -1;
    gf.xy(agg_fine_site(gf, gc, B, hc, i), x, y);
    agg_member(gf, gc, B, gf.nb(x, y, d), hj, mj);
    for (int c = 0; c < 9; ++c)
      if (gc.nb(xc, yc, c) == hj) {
        dc = c;
        break;
      }
    tab[e] = dc < 0 ? -1 : (dc << 8) | mj;
  }
  __syncthreads();
  for (int e = tid; e < 9 * K2 * K2; e += blockDim.x) {
    int dc = e / (K2 * K2), r = (e / K2) % K2, c = e % K2;
    int s = r / k, kap = r % k, t = c / k, lam = c % k;
    zd acc = mk(0.0, 0.0);
    for (int i = 0; i < M; ++i) {
      zd qi = Qs[((4 * 2 + s) * M + i) * k + kap];  // the coarse site itself is offset 4
      for (int d = 0; d < 9; ++d) {
        int tb = tab[i * 9 + d];
        if (tb < 0 || (tb >> 8) != dc) continue;
        zd qj = Qs[((dc * 2 + t) * M + (tb & 255)) * k + lam];
        acc = acc + cmulc(qi, As[i * 36 + d * 4 + s * 2 + t] * qj);
      }
    }
    Ac[(long)hc * 9 * K2 * K2 + e] = acc;
  }
}

// ------------------------------------------------------ restrict / prolong
// fc[r][hc][s k + kappa] = sum_m conj(Q[hc][s][m][kappa]) r[r][fine(hc, m)][s]  (ABI layouts)
__global__ void k_agg_restrict(Geo gf, Geo gc, int B, int k, const zd *__restrict__ Q, const zd *__restrict__ rv,
                               zd *__restrict__ fc, int nrhs) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int nc = gc.nsites(), K2 = 2 * k, M = B * B;
  if (t >= (long)nrhs * nc * K2) return;
  int v = (int)(t % K2), hc = (int)((t / K2) % nc), r = (int)(t / ((long)K2 * nc));
  int s = v / k, kap = v % k;
  const zd *rr = rv + (long)r * gf.nsites() * 2;
  zd acc = mk(0.0, 0.0);
  for (int m = 0; m < M; ++m)
    acc = acc + cmulc(Q[(((long)hc * 2 + s) * M + m) * k + kap], rr[2 * (long)agg_fine_site(gf, gc, B, hc, m) + s]);
  fc[t] = acc;
}

// x[r][h][s] += sum_kappa Q[hc][s][m][kappa] e[r][hc][s k + kappa]
__global__ void k_agg_prolong(Geo gf, Geo gc, int B, int k, const zd *__restrict__ Q, const zd *__restrict__ e,
                              zd *__restrict__ x, int nrhs) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int nf = gf.nsites(), K2 = 2 * k, M = B * B;
  if (t >= (long)nrhs * nf * 2) return;
  int s = (int)(t & 1), h = (int)((t >> 1) % nf), r = (int)(t / (2L * nf));
  int hc, m;
  agg_member(gf, gc, B, h, hc, m);
  const zd *er = e + ((long)r * gc.nsites() + hc) * K2 + s * k;
  zd acc = mk(0.0, 0.0);
  for (int kap = 0; kap < k; ++kap) acc = acc + Q[(((long)hc * 2 + s) * M + m) * k + kap] * er[kap];
  x[t] = x[t] + acc;
}

// ABI [nrhs][nc][K2] (complex128) <-> internal [nc][nrhs][K2] in T
template <typename T>
__global__ void k_agg_in(const zd *__restrict__ src, cx<T> *__restrict__ dst, int nc, int nrhs, int K2) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)nc * nrhs * K2) return;
  int v = (int)(t % K2), r = (int)((t / K2) % nrhs), h = (int)(t / ((long)K2 * nrhs));
  dst[t] = ccast<T>(src[((long)r * nc + h) * K2 + v]);
}
template <typename T>
__global__ void k_agg_out(const cx<T> *__restrict__ src, zd *__restrict__ dst, int nc, int nrhs, int K2) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)nc * nrhs * K2) return;
  int v = (int)(t % K2), h = (int)((t / K2) % nc), r = (int)(t / ((long)K2 * nc));
  dst[t] = widen<double>(src[((long)h * nrhs + r) * K2 + v]);
}

__global__ void k_agg_to_f32(const zd *__restrict__ a, zf *__restrict__ b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = ccast<float>(a[i]);
}

// deterministic filler for timing buffers (values in [-1, 1))
__global__ void k_agg_fill(float *v, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (float)((i * 2654435761ull) & 0xffff) * (1.0f / 32768.f) - 1.0f;
}

// ------------------------------------------------- apply on CUDA cores
// one block of 64 threads per (coarse site, chunk of 64 right-hand sides);
// the site's nine blocks in shared memory; thread r computes y_r (K2 complex
// values), in the order d, then j, of the oracle's definition
template <typename T, int K2>
__global__ void __launch_bounds__(64) k_agg_apply_simt(Geo gc, const cx<T> *__restrict__ Ac,
                                                       const cx<T> *__restrict__ X, cx<T> *__restrict__ Y,
                                                       int nrhs) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cx<T> *As = (cx<T> *)sm_raw;  // [9][K2][K2]
  int h = blockIdx.x, r = blockIdx.y * 64 + threadIdx.x;
  for (int e = threadIdx.x; e < 9 * K2 * K2; e += 64) As[e] = Ac[(long)h * 9 * K2 * K2 + e];
  __syncthreads();
  if (r >= nrhs) return;
  int x0, y0;
  gc.xy(h, x0, y0);
  cx<T> acc[K2];
#pragma unroll
  for (int c = 0; c < K2; ++c) acc[c] = mk<T>(0, 0);
  for (int d = 0; d < 9; ++d) {
    const cx<T> *xr = X + ((long)gc.nb(x0, y0, d) * nrhs + r) * K2;
    const cx<T> *Ad = As + d * K2 * K2;
#pragma unroll 2
    for (int j = 0; j < K2; j += 2) {
      cx<T> xj[2];
      if constexpr (sizeof(T) == 4) {
        float4 v = __ldg((const float4 *)(xr + j));
        xj[0] = mk((T)v.x, (T)v.y);
        xj[1] = mk((T)v.z, (T)v.w);
      } else {
        xj[0] = xr[j];
        xj[1] = xr[j + 1];
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int c = 0; c < K2; ++c) cfma(acc[c], Ad[c * K2 + j + u], xj[u]);
    }
  }
  cx<T> *yr = Y + ((long)h * nrhs + r) * K2;
#pragma unroll
  for (int c = 0; c < K2; ++c) yr[c] = acc[c];
}

// ------------------------------------------------- apply on tensor cores
#define AGG_TC_K2 16

// TF32 value nearest to v (the 10 explicit mantissa bits kept, ties away from zero)
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xffffe000u);
}

// shared-memory operand descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3ffffu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t ta, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(ta),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
      "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]),
      "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]),
      "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mb) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
}

// Warp-specialised persistent kernel, one block per SM (all 512 tensor-memory
// columns), 13 warps: warps 4-7 and 8-11 are two producer groups that build
// the even and odd steps (a step = one offset d of one coarse site: the 128
// A rows into tensor memory, the 16 x 16 stencil block hi and lo into shared
// memory); warp 12 issues the MMAs; warps 0-3 drain the accumulators.  Warp
// w reaches tensor-memory lanes 32 (w mod 4) .. +31, so every group of four
// covers the 128 rows.  Six stages (tensor-memory columns 64 s .. 64 s + 63:
// A hi, A lo) and two accumulator sets (columns 384 + 64 a: hi*hi of the three
// rows of offsets, then the corrections) are handed over by mbarriers:
// full[s] (128 producer arrivals), empty[s] (MMA commit), accfull[a] (MMA
// commit at a site's last step), accempty[a] (128 epilogue arrivals).  Every
// wait is bounded by a one-second timer; on a timeout the status word is set
// and the waiting role stops, so the others run into their own bounded waits
// and the block reaches its final barrier, frees tensor memory and returns.
#define AGG_TC_STAGES 6
#define AGG_TC_THREADS (13 * 32)
// TERMS = 3: hi*hi + hi*lo + lo*hi (FP32 accuracy); TERMS = 1: hi*hi only
// (TF32 operands, about 1e-3 relative: no lo parts are built or multiplied)
template <int TERMS>
__global__ void __launch_bounds__(AGG_TC_THREADS, 1) k_agg_apply_tc(Geo gc, const zf *__restrict__ Ac,
                                                                    const zf *__restrict__ X, zf *__restrict__ Y,
                                                                    int nrhs, int *flag) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  const int S = AGG_TC_STAGES;
  float *Bs = (float *)sm;  // [stage][hi, lo][16 rows][32 floats], 128-byte swizzle
  uint64_t *bars = (uint64_t *)(sm + S * 2 * 16 * 128);
  uint64_t *full = bars, *empty = bars + S, *accfull = bars + 2 * S, *accempty = bars + 2 * S + 2;
  uint32_t *tslot = (uint32_t *)(bars + 2 * S + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nc = gc.nsites(), r0 = blockIdx.y * 64;
  const unsigned long long LIMIT = 1000000000ull;
  const int nsite = blockIdx.x < nc ? (nc - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nstep = 9 * nsite;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full[i]), 128);
      mbar_init(smem_u32(&empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&accfull[i]), 1);
      mbar_init(smem_u32(&accempty[i]), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tb = *tslot, lane_off = (uint32_t)(32 * (warp & 3)) << 16;
  bool ok = true;
  if (warp >= 4 && warp < 12) {
    // ---------------------------------------------------------- producers
    const int g = (warp - 4) >> 2;                    // steps g, g + 2, g + 4, ...
    const int R = 32 * (warp & 3) + lane, rr = R >> 1, p = R & 1;
    const bool rvalid = r0 + rr < nrhs;
    const int t128 = tid - 128 * (1 + g);             // 0..127 inside the group
    const int cb = t128 >> 3, qb = t128 & 7;          // B chunk: row cb, 16-byte chunk qb
    // the two threads of a right-hand side (rows 2 rr, 2 rr + 1) each load and
    // split half of its 16 complex values (p = 0: variables 0-7, p = 1: 8-15)
    // and trade halves by shuffles, so every value is split once per step
    auto load_step = [&](int s, float4 (&xv)[4], float4 &bv) {
      if (s >= nstep) return;
      int h = blockIdx.x + (s / 9) * gridDim.x, d = s % 9, xs, ys;
      gc.xy(h, xs, ys);
      if (rvalid) {
        const float4 *src = (const float4 *)(X + ((long)gc.nb(xs, ys, d) * nrhs + r0 + rr) * AGG_TC_K2) + 4 * p;
#pragma unroll
        for (int q = 0; q < 4; ++q) xv[q] = __ldg(src + q);
      }
      bv = __ldg((const float4 *)(Ac + (((long)h * 9 + d) * AGG_TC_K2 + cb) * AGG_TC_K2) + qb);
    };
    float4 xv[4], bv = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) xv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    load_step(g, xv, bv);
    for (int s = g; s < nstep; s += 2) {
      float4 xn[4], bn = bv;
#pragma unroll
      for (int q = 0; q < 4; ++q) xn[q] = xv[q];
      load_step(s + 2, xn, bn);
      const int st = s % S;
      if (s >= S) {  // the vote keeps the warp converged for the .sync.aligned tensor-memory stores
        if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&empty[st]), (uint32_t)(((s / S) - 1) & 1), LIMIT))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      // row R of A: hi parts to columns 0-31 of the stage, then lo parts to 32-63;
      // row 2r holds (Re x_j, -Im x_j), row 2r + 1 (Im x_j, Re x_j), j = 0..15
#pragma unroll
      for (int part = 0; part < (TERMS == 3 ? 2 : 1); ++part) {
        float own[16], oth[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float v[4] = {xv[q].x, xv[q].y, xv[q].z, xv[q].w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float hi = tf32_rn(v[u]);
            own[4 * q + u] = rvalid ? (part ? tf32_rn(v[u] - hi) : hi) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) oth[u] = __shfl_xor_sync(0xffffffffu, own[u], 1);
        float av[32];
#pragma unroll
        for (int j = 0; j < 16; ++j) {  // variable j: element 2 (j mod 8) (re), + 1 (im) of its half
          const float re = (j < 8) == (p == 0) ? own[2 * (j & 7)] : oth[2 * (j & 7)];
          const float im = (j < 8) == (p == 0) ? own[2 * (j & 7) + 1] : oth[2 * (j & 7) + 1];
          av[2 * j] = p ? im : re;
          av[2 * j + 1] = p ? re : -im;
        }
        tmem_st32(tb + lane_off + st * 64 + 32 * part, av);
      }
      {
        float4 v = bv;
        float4 hi = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
        float4 lo = make_float4(tf32_rn(v.x - hi.x), tf32_rn(v.y - hi.y), tf32_rn(v.z - hi.z), tf32_rn(v.w - hi.w));
        int off = cb * 32 + ((qb ^ (cb & 7)) * 4);
        *(float4 *)(Bs + (st * 2 + 0) * 512 + off) = hi;
        if (TERMS == 3) *(float4 *)(Bs + (st * 2 + 1) * 512 + off) = lo;
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&full[st]));
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = xn[q];
      bv = bn;
    }
  } else if (warp == 12) {
    // ------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(AGG_TC_K2 >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      for (int s = 0; s < nstep && ok; ++s) {
        const int st = s % S, i = s / 9, d = s % 9, a = i & 1;
        if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((s / S) & 1), LIMIT)) {
          ok = false;
          break;
        }
        if (d == 0 && i >= 2 && !mbar_wait(smem_u32(&accempty[a]), (uint32_t)(((i >> 1) - 1) & 1), LIMIT)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t bh = smem_u32(Bs + (st * 2 + 0) * 512), bl = smem_u32(Bs + (st * 2 + 1) * 512);
        const uint32_t ah = tb + st * 64, al = ah + 32;
        const uint32_t tG = tb + 384 + 64 * a + 16 * (d / 3), tC = tb + 384 + 64 * a + 48;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          tc_mma_tf32(tG, ah + 8 * ks, smem_desc_sw128(bh + 32 * ks), idesc, (d % 3 > 0 || ks > 0) ? 1u : 0u);
          if (TERMS == 3) {
            tc_mma_tf32(tC, ah + 8 * ks, smem_desc_sw128(bl + 32 * ks), idesc, (d > 0 || ks > 0) ? 1u : 0u);
            tc_mma_tf32(tC, al + 8 * ks, smem_desc_sw128(bh + 32 * ks), idesc, 1u);
          }
        }
        tc_commit(smem_u32(&empty[st]));
        if (d == 8) tc_commit(smem_u32(&accfull[a]));
      }
      if (!ok) {
        atomicExch(flag, 2);
      } else if (nstep > 0) {  // nothing may be in flight when tensor memory is freed
        const int last = nstep - 1;
        if (!mbar_wait(smem_u32(&empty[last % S]), (uint32_t)((last / S) & 1), LIMIT)) atomicExch(flag, 2);
      }
    }
  } else if (warp < 4) {
    // --------------------------------------------------------- epilogue
    const int R = 32 * warp + lane, rr = R >> 1, p = R & 1;
    const bool rvalid = r0 + rr < nrhs;
    for (int i = 0; i < nsite; ++i) {
      const int a = i & 1, h = blockIdx.x + i * gridDim.x;
      if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&accfull[a]), (uint32_t)((i >> 1) & 1), LIMIT))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float y[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) y[c] = 0.f;
#pragma unroll
      for (int b = 0; b < (TERMS == 3 ? 4 : 3); ++b) {  // ((D0 + D1) + D2) + corrections
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tb + 384 + 64 * a + 16 * b + lane_off)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 16; ++c) y[c] = __fadd_rn(y[c], __uint_as_float(v[c]));
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&accempty[a]));
      float other[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) other[c] = __shfl_xor_sync(0xffffffffu, y[c], 1);
      if (p == 0 && rvalid) {
        float4 *dst = (float4 *)(Y + ((long)h * nrhs + r0 + rr) * AGG_TC_K2);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(y[2 * q], other[2 * q], y[2 * q + 1], other[2 * q + 1]);
      }
    }
  }
  if (!ok) atomicExch(flag, 2);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(512) : "memory");
  }
}

// ------------------------------------------------------------------ host
namespace {
int agg_check_level(wl_amg *amg, int level, int B, int k) {
  if (!amg || level < 0 || level >= amg->L) return WL_EINVAL;
  int N = amg->lev[level].N;
  if ((B != 2 && B != 4) || N % B || (N / 2) % B || N / B < 8 || k < 1 || k > 16 || k > B * B) return WL_EINVAL;
  return WL_OK;
}

wl_agg *agg_new(wl_amg *amg, int level, int B, int k) {
  wl_agg *g = new wl_agg();
  g->amg = amg;
  g->level = level;
  g->B = B;
  g->k = k;
  g->M = B * B;
  g->Nf = amg->lev[level].N;
  g->Nc = g->Nf / B;
  g->gf = make_geo(g->Nf);
  g->gc = make_geo(g->Nc);
  g->nf = g->gf.nsites();
  g->nc = g->gc.nsites();
  g->cap = g->cap64 = 0;
  wl::amg_retain(amg);
  return g;
}

void agg_free(wl_agg *g) {
  if (!g) return;
  g->Q.release();
  g->Ac.release();
  g->Ac32.release();
  g->X.release();
  g->Y.release();
  g->X64.release();
  g->Y64.release();
  g->flag.release();
  wl::amg_release(g->amg);
  delete g;
}

int agg_alloc(wl_agg *g) {
  size_t K2 = 2 * (size_t)g->k;
  WL_TRY(g->Q.alloc(sizeof(zd) * (size_t)g->nc * 2 * g->M * g->k));
  WL_TRY(g->Ac.alloc(sizeof(zd) * (size_t)g->nc * 9 * K2 * K2));
  WL_TRY(g->Ac32.alloc(sizeof(zf) * (size_t)g->nc * 9 * K2 * K2));
  WL_TRY(g->flag.alloc(sizeof(int)));
  return WL_OK;
}

int agg_finish(wl_agg *g, cudaStream_t s) {
  long n = (long)g->nc * 9 * 4 * g->k * g->k;
  k_agg_to_f32<<<WL_GRID(n, 256), 256, 0, s>>>(g->Ac.as<zd>(), g->Ac32.as<zf>(), n);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

int agg_buffers(wl_agg *g, int nrhs, int fp64) {
  size_t n = (size_t)g->nc * nrhs * 2 * g->k;
  if (fp64) {
    if (nrhs > g->cap64) {
      WL_TRY(g->X64.alloc(sizeof(zd) * n));
      WL_TRY(g->Y64.alloc(sizeof(zd) * n));
      g->cap64 = nrhs;
    }
  } else if (nrhs > g->cap) {
    WL_TRY(g->X.alloc(sizeof(zf) * n));
    WL_TRY(g->Y.alloc(sizeof(zf) * n));
    g->cap = nrhs;
  }
  return WL_OK;
}

template <typename T, int K2>
int launch_simt(wl_agg *g, const cx<T> *Ac, const cx<T> *X, cx<T> *Y, int nrhs, cudaStream_t s) {
  size_t smem = sizeof(cx<T>) * 9 * K2 * K2;
  static std::atomic<unsigned long long> limit_set{0};
  int dev = 0;
  WL_CUDA(cudaGetDevice(&dev));
  if (!(limit_set.load() & (1ull << (dev & 63)))) {
    WL_CUDA(cudaFuncSetAttribute((const void *)k_agg_apply_simt<T, K2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    limit_set.fetch_or(1ull << (dev & 63));
  }
  dim3 grid(g->nc, (nrhs + 63) / 64);
  k_agg_apply_simt<T, K2><<<grid, 64, smem, s>>>(g->gc, Ac, X, Y, nrhs);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

// dynamic shared memory of the tensor-core kernel: six B stages (24 KB), the
// mbarriers and the tensor-memory slot, 1 KB of alignment slack; 120 KB are
// asked for so that one block holds an SM (it allocates all 512
// tensor-memory columns)
const size_t TC_SMEM = 120 * 1024;

template <int TERMS>
int launch_tc(wl_agg *g, const zf *X, zf *Y, int nrhs, cudaStream_t s) {
  static std::atomic<unsigned long long> limit_set{0};
  int dev = 0;
  WL_CUDA(cudaGetDevice(&dev));
  if (!(limit_set.load() & (1ull << (dev & 63)))) {
    WL_CUDA(cudaFuncSetAttribute((const void *)k_agg_apply_tc<TERMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TC_SMEM));
    limit_set.fetch_or(1ull << (dev & 63));
  }
  int nsm = 0;
  WL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  dim3 grid(std::min(g->nc, nsm), (nrhs + 63) / 64);
  k_agg_apply_tc<TERMS><<<grid, AGG_TC_THREADS, TC_SMEM, s>>>(g->gc, g->Ac32.as<zf>(), X, Y, nrhs,
                                                                g->flag.as<int>());
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return WL_OK;
}

int apply_internal(wl_agg *g, int kernel, int nrhs, cudaStream_t s) {
  int K2 = 2 * g->k;
  if (kernel == WL_AGG_TC) return launch_tc<3>(g, g->X.as<zf>(), g->Y.as<zf>(), nrhs, s);
  if (kernel == WL_AGG_TC1) return launch_tc<1>(g, g->X.as<zf>(), g->Y.as<zf>(), nrhs, s);
  if (kernel == WL_AGG_FP32) {
    const zf *A = g->Ac32.as<zf>();
    if (K2 == 8) return launch_simt<float, 8>(g, A, g->X.as<zf>(), g->Y.as<zf>(), nrhs, s);
    if (K2 == 16) return launch_simt<float, 16>(g, A, g->X.as<zf>(), g->Y.as<zf>(), nrhs, s);
    return launch_simt<float, 32>(g, A, g->X.as<zf>(), g->Y.as<zf>(), nrhs, s);
  }
  const zd *A = g->Ac.as<zd>();
  if (K2 == 8) return launch_simt<double, 8>(g, A, g->X64.as<zd>(), g->Y64.as<zd>(), nrhs, s);
  if (K2 == 16) return launch_simt<double, 16>(g, A, g->X64.as<zd>(), g->Y64.as<zd>(), nrhs, s);
  return launch_simt<double, 32>(g, A, g->X64.as<zd>(), g->Y64.as<zd>(), nrhs, s);
}

int check_apply_args(wl_agg *g, int nrhs, int kernel) {
  bool tc = kernel == WL_AGG_TC || kernel == WL_AGG_TC1;
  if (!g || nrhs < 1 || nrhs > 4096 || (kernel != WL_AGG_FP64 && kernel != WL_AGG_FP32 && !tc)) {
    wl_set_error("agg_apply: invalid argument (1 <= nrhs <= 4096, kernel WL_AGG_FP64 / FP32 / TC / TC1)");
    return WL_EINVAL;
  }
  if (!tc && g->k != 4 && g->k != 8 && g->k != 16) {
    wl_set_error("agg_apply: the block-stencil apply takes k = 4, 8 or 16");
    return WL_EINVAL;
  }
  if (tc && g->k != 8) {
    wl_set_error("agg_apply: the tensor-core apply takes k = 8 (16 x 16 blocks)");
    return WL_EINVAL;
  }
  return WL_OK;
}

int read_flag(wl_agg *g, cudaStream_t s, int *out) {
  WL_CUDA(cudaMemcpyAsync(out, g->flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}
}  // namespace

extern "C" int agg_create(wl_amg *amg, int level, int B, int k, const void *V, wl_agg **out) {
  if (!out || !V || agg_check_level(amg, level, B, k)) {
    wl_set_error("agg_create: invalid argument (B = 2 or 4 dividing N_l / 2, N_l / B >= 8, 1 <= k <= min(16, B^2))");
    return WL_EINVAL;
  }
  WL_TRY(wl::enter(amg->op));
  cudaStream_t s = amg->op->stream;
  wl_agg *g = agg_new(amg, level, B, k);
  int rc = agg_alloc(g);
  if (!rc && cudaMemsetAsync(g->flag.p, 0, sizeof(int), s) != cudaSuccess) rc = WL_ECUDA;
  if (!rc) {
    long tasks = 2L * g->nc;
    size_t smem = sizeof(zd) * 4 * 32 * k;
    k_agg_interp<<<WL_GRID(tasks, 4), 128, smem, s>>>(g->gf, g->gc, B, k, (const zd *)V, 2L * g->nf, g->Q.as<zd>(),
                                                      g->flag.as<int>());
    size_t gsm = sizeof(zd) * (9 * 2 * g->M * k + g->M * 36) + sizeof(int) * g->M * 9;
    if (gsm > 48 * 1024 &&
        cudaFuncSetAttribute((const void *)k_agg_galerkin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm) !=
            cudaSuccess)
      rc = WL_ECUDA;
    if (!rc) {
      k_agg_galerkin<<<g->nc, 256, gsm, s>>>(g->gf, g->gc, B, k, amg->lev[level].op64.A.as<zd>(), g->Q.as<zd>(),
                                             g->Ac.as<zd>());
      wl_count_launches(2);
      if (cudaGetLastError() != cudaSuccess) rc = WL_ECUDA;
    }
  }
  if (!rc) rc = agg_finish(g, s);
  int bad = 0;
  if (!rc) rc = read_flag(g, s, &bad);
  if (!rc && bad) {
    wl_set_error("agg_create: the test vectors restricted to some aggregate and spin have rank < %d", k);
    rc = WL_EINVAL;
  }
  if (rc) {
    agg_free(g);
    return rc;
  }
  *out = g;
  return WL_OK;
}

extern "C" int agg_import(wl_amg *amg, int level, int B, int k, const void *Q, const void *Ac, wl_agg **out) {
  if (!out || !Q || !Ac || agg_check_level(amg, level, B, k)) {
    wl_set_error("agg_import: invalid argument");
    return WL_EINVAL;
  }
  WL_TRY(wl::enter(amg->op));
  cudaStream_t s = amg->op->stream;
  wl_agg *g = agg_new(amg, level, B, k);
  int rc = agg_alloc(g);
  if (!rc && (cudaMemcpyAsync(g->Q.p, Q, g->Q.bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
              cudaMemcpyAsync(g->Ac.p, Ac, sizeof(zd) * (size_t)g->nc * 9 * 4 * k * k, cudaMemcpyDeviceToDevice, s) !=
                  cudaSuccess ||
              cudaMemsetAsync(g->flag.p, 0, sizeof(int), s) != cudaSuccess))
    rc = WL_ECUDA;
  if (!rc) rc = agg_finish(g, s);
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = WL_ECUDA;
  if (rc) {
    agg_free(g);
    return rc;
  }
  *out = g;
  return WL_OK;
}

extern "C" int agg_export(wl_agg *g, void *Q, void *Ac) {
  if (!g || !Q || !Ac) return WL_EINVAL;
  WL_TRY(wl::enter(g->amg->op));
  cudaStream_t s = g->amg->op->stream;
  WL_CUDA(cudaMemcpyAsync(Q, g->Q.p, sizeof(zd) * (size_t)g->nc * 2 * g->M * g->k, cudaMemcpyDeviceToDevice, s));
  WL_CUDA(cudaMemcpyAsync(Ac, g->Ac.p, sizeof(zd) * (size_t)g->nc * 9 * 4 * g->k * g->k, cudaMemcpyDeviceToDevice, s));
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

extern "C" int agg_info(wl_agg *g, int *nc, int *Nc, int *k) {
  if (!g) return WL_EINVAL;
  if (nc) *nc = g->nc;
  if (Nc) *Nc = g->Nc;
  if (k) *k = g->k;
  return WL_OK;
}

extern "C" void agg_destroy(wl_agg *g) { agg_free(g); }

extern "C" int agg_apply(wl_agg *g, const void *x, void *y, int nrhs, int kernel) {
  WL_TRY(check_apply_args(g, nrhs, kernel));
  if (!x || !y) return WL_EINVAL;
  WL_TRY(wl::enter(g->amg->op));
  cudaStream_t s = g->amg->op->stream;
  int K2 = 2 * g->k, fp64 = kernel == WL_AGG_FP64;
  WL_TRY(agg_buffers(g, nrhs, fp64));
  long n = (long)g->nc * nrhs * K2;
  WL_CUDA(cudaMemsetAsync(g->flag.p, 0, sizeof(int), s));
  if (fp64) k_agg_in<double><<<WL_GRID(n, 256), 256, 0, s>>>((const zd *)x, g->X64.as<zd>(), g->nc, nrhs, K2);
  else k_agg_in<float><<<WL_GRID(n, 256), 256, 0, s>>>((const zd *)x, g->X.as<zf>(), g->nc, nrhs, K2);
  wl_count_launches(1);
  WL_TRY(apply_internal(g, kernel, nrhs, s));
  if (fp64) k_agg_out<double><<<WL_GRID(n, 256), 256, 0, s>>>(g->Y64.as<zd>(), (zd *)y, g->nc, nrhs, K2);
  else k_agg_out<float><<<WL_GRID(n, 256), 256, 0, s>>>(g->Y.as<zf>(), (zd *)y, g->nc, nrhs, K2);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  int bad = 0;
  WL_TRY(read_flag(g, s, &bad));
  if (bad) {
    wl_set_error("agg_apply: a tensor-core wait ran out of time (status %d)", bad);
    return WL_TIMEOUT;
  }
  return WL_OK;
}

extern "C" int agg_restrict(wl_agg *g, const void *r, void *fc, int nrhs) {
  if (!g || !r || !fc || nrhs < 1) return WL_EINVAL;
  WL_TRY(wl::enter(g->amg->op));
  cudaStream_t s = g->amg->op->stream;
  long n = (long)nrhs * g->nc * 2 * g->k;
  k_agg_restrict<<<WL_GRID(n, 256), 256, 0, s>>>(g->gf, g->gc, g->B, g->k, g->Q.as<zd>(), (const zd *)r, (zd *)fc,
                                                 nrhs);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

extern "C" int agg_prolong(wl_agg *g, const void *e, void *x, int nrhs) {
  if (!g || !e || !x || nrhs < 1) return WL_EINVAL;
  WL_TRY(wl::enter(g->amg->op));
  cudaStream_t s = g->amg->op->stream;
  long n = (long)nrhs * g->nf * 2;
  k_agg_prolong<<<WL_GRID(n, 256), 256, 0, s>>>(g->gf, g->gc, g->B, g->k, g->Q.as<zd>(), (const zd *)e, (zd *)x,
                                                nrhs);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  WL_CUDA(cudaStreamSynchronize(s));
  return WL_OK;
}

extern "C" int agg_time_apply(wl_agg *g, int nrhs, int kernel, int reps, double *avg_ms) {
  WL_TRY(check_apply_args(g, nrhs, kernel));
  if (reps < 1 || !avg_ms) return WL_EINVAL;
  WL_TRY(wl::enter(g->amg->op));
  cudaStream_t s = g->amg->op->stream;
  int fp64 = kernel == WL_AGG_FP64;
  WL_TRY(agg_buffers(g, nrhs, fp64));
  long n = (long)g->nc * nrhs * 2 * g->k * 2 * (fp64 ? 2 : 1);  // floats (or float pairs of a double)
  k_agg_fill<<<WL_GRID(n, 256), 256, 0, s>>>(fp64 ? (float *)g->X64.p : (float *)g->X.p, fp64 ? n / 2 : n);
  if (fp64) WL_CUDA(cudaMemsetAsync(g->X64.p, 0, g->X64.bytes, s));  // keep the doubles finite
  WL_CUDA(cudaMemsetAsync(g->flag.p, 0, sizeof(int), s));
  WL_TRY(apply_internal(g, kernel, nrhs, s));
  cudaEvent_t e0, e1;
  WL_CUDA(cudaEventCreate(&e0));
  WL_CUDA(cudaEventCreate(&e1));
  int rc = WL_OK;
  if (cudaEventRecord(e0, s) != cudaSuccess) rc = WL_ECUDA;
  for (int i = 0; i < reps && !rc; ++i) rc = apply_internal(g, kernel, nrhs, s);
  float ms = 0;
  if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = WL_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  int bad = 0;
  WL_TRY(read_flag(g, s, &bad));
  if (bad) {
    wl_set_error("agg_time_apply: a tensor-core wait ran out of time");
    return WL_TIMEOUT;
  }
  *avg_ms = (double)ms / reps;
  return WL_OK;
}
