// wl_hier.cu -- hierarchy objects: import / export of the hierarchy file,
// per-precision operator copies, Kaczmarz denominators, the FP64 inverse of
// the coarsest operator (Sec. 4: the N = 16 grid is solved directly), and
// workspace management.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "wl_common.cuh"

namespace wl {
uint64_t hash_bytes(const void *p, size_t n);
}

static const char kMagic[8] = {'W', 'L', 'A', 'M', 'G', 'H', '0', '1'};

extern "C" void amg_params_default(amg_params *p) {
  memset(p, 0, sizeof(*p));
  p->levels = 0;  // 0: derive from L (4x4 cells while the next grid keeps N >= 16, then 2x2)
  p->k_r = 8;
  p->k_e = 8;
  p->setup_mu[0] = 10;
  p->setup_mu[1] = 5;
  p->nu_pre = 2;
  p->nu_post = 2;
  p->omega = 1.0;
  p->cycle = WL_CYCLE_V;
  p->fgmres_m = 20;
  p->max_restarts = 50;
  p->precision = WL_FP64;
  p->seed = 1;
  p->gs_passes = 2;
  p->zero_guess = 0;
}

namespace wl {

// resolve levels / blocks for lattice side N; fills Nl[]
int resolve_levels(int N, amg_params *p, int *Nl) {
  if (p->levels == 0) {
    int n = N, L = 1;
    while (n > 16) {
      int b = (n / 4 >= 16) ? 4 : 2;
      p->block[L - 1] = b;
      n /= b;
      L++;
    }
    p->levels = L;
  }
  if (p->levels < 2 || p->levels > 8) {
    wl_set_error("levels = %d must be in [2, 8]", p->levels);
    return WL_EINVAL;
  }
  Nl[0] = N;
  for (int l = 0; l + 1 < p->levels; ++l) {
    int B = p->block[l];
    if ((B != 2 && B != 4) || Nl[l] % 8 || (Nl[l] / 2) % B) {
      wl_set_error("block[%d] = %d incompatible with N_l = %d (need B in {2,4}, N_l %% 8 == 0)", l, B,
                   Nl[l]);
      return WL_EINVAL;
    }
    Nl[l + 1] = Nl[l] / B;
  }
  if (Nl[p->levels - 1] < 4) {
    wl_set_error("coarsest grid N = %d too small", Nl[p->levels - 1]);
    return WL_EINVAL;
  }
  if (p->fgmres_m < 1 || p->fgmres_m > 32 || p->max_restarts < 1 || p->nu_pre < 0 ||
      p->nu_post < 0 || p->gs_passes < 1 || p->gs_passes > 2 || p->sweep_kernel < 0 || p->sweep_kernel > 2 ||
      p->kacz_order < 0 || p->kacz_order > 1 || p->arnoldi_matvec < 0 || p->arnoldi_matvec > 1 ||
      p->setup_cycle < 0 || p->setup_cycle > 1 || p->gs_arith < 0 || p->gs_arith > 1 ||
      (p->gs_arith == 1 && (p->precision == WL_FP64 || p->arnoldi_matvec != 1)) ||
      (p->precision != WL_FP64 && p->precision != WL_FP32 && p->precision != WL_FP32_BF16) ||
      (p->cycle != WL_CYCLE_V && p->cycle != WL_CYCLE_W)) {
    wl_set_error("invalid solve parameters");
    return WL_EINVAL;
  }
  return WL_OK;
}

}  // namespace wl

// ------------------------------------------------------------- conversions
__global__ void k_to_f32(const zd *__restrict__ a, zf *__restrict__ b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = ccast<float>(a[i]);
}
__global__ void k_to_bf16(const zd *__restrict__ a, zb *__restrict__ b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i].v = __floats2bfloat162_rn((float)a[i].re, (float)a[i].im);
}
__global__ void k_d_to_f(const double *__restrict__ a, float *__restrict__ b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_den_bf16(int n, const zb *__restrict__ A, float *__restrict__ den) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * n) return;
  int h = tid >> 1, t = tid & 1;
  float s = 0;
  for (int d = 0; d < 9; ++d)
    for (int u = 0; u < 2; ++u) {
      float2 f = __bfloat1622float2(A[((long)h * 9 + d) * 4 + t * 2 + u].v);
      s += f.x * f.x + f.y * f.y;
    }
  den[tid] = s;
}

// Gauss-Jordan inversion with partial pivoting, one block; M is overwritten
// by junk, Inv receives M^-1 (both row major, n x n complex double).
__global__ void __launch_bounds__(1024) k_gauss_jordan(int n, zd *M, zd *Inv, int *status) {
  extern __shared__ unsigned char smem_raw[];
  zd *fac = (zd *)smem_raw;                 // [n]
  double *bv = (double *)(fac + n);          // [blockDim]
  int *bi = (int *)(bv + blockDim.x);        // [blockDim]
  int tid = threadIdx.x, nt = blockDim.x;
  for (long i = tid; i < (long)n * n; i += nt) Inv[i] = mk((i / n == i % n) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bidx = k;
    for (int i = k + tid; i < n; i += nt) {
      double v = cnorm2(M[(long)i * n + k]);
      if (v > best) {
        best = v;
        bidx = i;
      }
    }
    bv[tid] = best;
    bi[tid] = bidx;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s && (bv[tid + s] > bv[tid] || (bv[tid + s] == bv[tid] && bi[tid + s] < bi[tid]))) {
        bv[tid] = bv[tid + s];
        bi[tid] = bi[tid + s];
      }
      __syncthreads();
    }
    int p = bi[0];
    if (bv[0] <= 0.0) {
      if (tid == 0) *status = 1;
      return;
    }
    if (p != k)
      for (int j = tid; j < n; j += nt) {
        zd t = M[(long)k * n + j];
        M[(long)k * n + j] = M[(long)p * n + j];
        M[(long)p * n + j] = t;
        t = Inv[(long)k * n + j];
        Inv[(long)k * n + j] = Inv[(long)p * n + j];
        Inv[(long)p * n + j] = t;
      }
    __syncthreads();
    zd piv = M[(long)k * n + k];
    double d = cnorm2(piv);
    zd ip = mk(piv.re / d, -piv.im / d);
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      M[(long)k * n + j] = ip * M[(long)k * n + j];
      Inv[(long)k * n + j] = ip * Inv[(long)k * n + j];
    }
    __syncthreads();
    for (int i = tid; i < n; i += nt) fac[i] = M[(long)i * n + k];
    __syncthreads();
    for (long q = tid; q < (long)n * n; q += nt) {
      int i = (int)(q / n), j = (int)(q % n);
      if (i == k) continue;
      zd f = fac[i];
      M[q] = M[q] - f * M[(long)k * n + j];
      Inv[q] = Inv[q] - f * Inv[(long)k * n + j];
    }
    __syncthreads();
  }
  if (tid == 0) *status = 0;
}

// dense coarsest operator from its stencil: M[(h,s),(nb(h,d),t)] += A[h][d][s][t]
__global__ void k_stencil_dense(Geo g, const zd *__restrict__ A, zd *M) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.nsites()) return;
  int n = 2 * g.nsites(), x, y;
  g.xy(h, x, y);
  for (int d = 0; d < 9; ++d) {
    int j = g.nb(x, y, d);
    for (int s = 0; s < 2; ++s)
      for (int t = 0; t < 2; ++t) {
        long o = (long)(2 * h + s) * n + 2 * j + t;
        M[o] = M[o] + A[((long)h * 9 + d) * 4 + s * 2 + t];
      }
  }
}

namespace wl {

int coarsest_invert(wl_amg *a) {
  cudaStream_t s = a->op->stream;
  Level &C = a->lev[a->L - 1];
  int n = 2 * C.n;
  a->nc = n;
  DBuf M, st;
  WL_TRY(M.alloc(sizeof(zd) * n * n));
  WL_TRY(st.alloc(sizeof(int)));
  WL_TRY(a->Ainv.alloc(sizeof(zd) * n * n));
  WL_TRY(a->Ainv32.alloc(sizeof(zf) * n * n));
  WL_CUDA(cudaMemsetAsync(M.p, 0, sizeof(zd) * n * n, s));
  k_stencil_dense<<<WL_GRID(C.n, 128), 128, 0, s>>>(C.geo, C.op64.A.as<zd>(), M.as<zd>());
  size_t sm = sizeof(zd) * n + (sizeof(double) + sizeof(int)) * 1024;
  WL_CUDA(cudaFuncSetAttribute(k_gauss_jordan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_gauss_jordan<<<1, 1024, sm, s>>>(n, M.as<zd>(), a->Ainv.as<zd>(), st.as<int>());
  WL_CUDA(cudaGetLastError());
  k_to_f32<<<WL_GRID((long)n * n, 256), 256, 0, s>>>(a->Ainv.as<zd>(), a->Ainv32.as<zf>(), (long)n * n);
  int hs = 1;
  WL_CUDA(cudaMemcpyAsync(&hs, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  WL_CUDA(cudaStreamSynchronize(s));
  M.release();
  st.release();
  if (hs) {
    wl_set_error("coarsest operator is singular");
    return WL_BAD_HIERARCHY;
  }
  return WL_OK;
}

// FP32 / BF16 copies and the Kaczmarz denominators of every level
int level_ops_build_copies(wl_amg *a) {
  cudaStream_t s = a->op->stream;
  for (int l = 0; l < a->L; ++l) {
    Level &L = a->lev[l];
    long na = (long)L.n * 36;
    WL_TRY(L.op64.den.alloc(sizeof(double) * L.n * 2));
    WL_TRY(compute_den64(L.N, L.op64.A.as<zd>(), L.op64.den.as<double>(), s));
    WL_TRY(L.op32.A.alloc(sizeof(zf) * na));
    WL_TRY(L.op32.den.alloc(sizeof(float) * L.n * 2));
    WL_TRY(L.opbf.A.alloc(sizeof(zb) * na));
    WL_TRY(L.opbf.den.alloc(sizeof(float) * L.n * 2));
    k_to_f32<<<WL_GRID(na, 256), 256, 0, s>>>(L.op64.A.as<zd>(), L.op32.A.as<zf>(), na);
    k_d_to_f<<<WL_GRID(2L * L.n, 256), 256, 0, s>>>(L.op64.den.as<double>(), L.op32.den.as<float>(), 2L * L.n);
    k_to_bf16<<<WL_GRID(na, 256), 256, 0, s>>>(L.op64.A.as<zd>(), L.opbf.A.as<zb>(), na);
    k_den_bf16<<<WL_GRID(2L * L.n, 256), 256, 0, s>>>(L.n, L.opbf.A.as<zb>(), L.opbf.den.as<float>());
    if (l + 1 < a->L) {
      long np = (long)L.n * 8;
      WL_TRY(L.op32.P.alloc(sizeof(zf) * np));
      WL_TRY(L.opbf.P.alloc(sizeof(zb) * np));
      k_to_f32<<<WL_GRID(np, 256), 256, 0, s>>>(L.op64.P.as<zd>(), L.op32.P.as<zf>(), np);
      k_to_bf16<<<WL_GRID(np, 256), 256, 0, s>>>(L.op64.P.as<zd>(), L.opbf.P.as<zb>(), np);
    }
    WL_CUDA(cudaGetLastError());
  }
  return WL_OK;
}

static void release_graphs(wl_amg *a) {
  for (auto &g : a->graphs) cudaGraphExecDestroy(g.exec);
  a->graphs.clear();
}

int ensure_workspace(wl_amg *a, int nrhs, int prec) {
  (void)prec;
  if (nrhs <= a->cap) return WL_OK;
  cudaStreamSynchronize(a->op->stream);
  release_graphs(a);
  int cap = std::max(nrhs, a->cap);
  for (int l = 0; l < a->L; ++l) {
    Level &L = a->lev[l];
    size_t vb = sizeof(zd) * (size_t)L.n * 2 * cap;
    WL_TRY(L.x.alloc(vb));
    WL_TRY(L.r.alloc(vb));
    WL_TRY(L.f.alloc(vb));
    WL_TRY(L.t.alloc(vb));
    DBuf *bs[4] = {&L.x, &L.r, &L.f, &L.t};
    for (auto *b : bs) WL_CUDA(cudaMemsetAsync(b->p, 0, vb, a->op->stream));
  }
  int m = a->prm.fgmres_m;
  size_t vb0 = sizeof(zd) * (size_t)a->lev[0].n * 2 * cap;
  WL_TRY(a->V.alloc(vb0 * (m + 1)));
  WL_TRY(a->Z.alloc(vb0 * m));
  WL_TRY(a->w.alloc(vb0));
  WL_TRY(a->bh.alloc(vb0));
  WL_TRY(a->xh.alloc(vb0));
  WL_TRY(a->rr.alloc(vb0));
  WL_CUDA(cudaMemsetAsync(a->V.p, 0, vb0 * (m + 1), a->op->stream));
  WL_CUDA(cudaMemsetAsync(a->Z.p, 0, vb0 * m, a->op->stream));
  WL_CUDA(cudaMemsetAsync(a->w.p, 0, vb0, a->op->stream));
  WL_TRY(a->red.alloc(sizeof(zd) * 1024 * (m + 2) * (size_t)cap));
  WL_TRY(a->small.alloc(sizeof(zd) * (size_t)cap * 8 * (m + 2) * (m + 2)));
  if (a->h_small) cudaFreeHost(a->h_small);
  a->h_small = nullptr;
  WL_CUDA(cudaMallocHost(&a->h_small, sizeof(double) * (size_t)cap * 16 + 64));
  a->cap = cap;
  return WL_OK;
}

// allocate the level structures for sizes Nl and copy P / coarse stencils
int hier_alloc(wl_amg *a, const int *Nl) {
  for (int l = 0; l < a->L; ++l) {
    Level &L = a->lev[l];
    L.N = Nl[l];
    L.B = (l + 1 < a->L) ? Nl[l] / Nl[l + 1] : 0;
    L.n = Nl[l] * Nl[l] / 2;
    L.geo = make_geo(Nl[l]);
    WL_TRY(L.op64.A.alloc(sizeof(zd) * (size_t)L.n * 36));
    if (l + 1 < a->L) WL_TRY(L.op64.P.alloc(sizeof(zd) * (size_t)L.n * 8));
  }
  return WL_OK;
}

int hier_finish(wl_amg *a) {
  WL_TRY(level_ops_build_copies(a));
  WL_TRY(coarsest_invert(a));
  WL_CUDA(cudaStreamSynchronize(a->op->stream));
  return WL_OK;
}

// The second solve lane of a: a hierarchy object whose operator data (links,
// level stencils, denominators, interpolation weights, coarsest inverse) are
// views of a's, with a stream, an event, a workspace and cycle graphs of its
// own.  Its operator's "caller" stream is a's work stream, so work queued on
// the twin first waits for everything queued on a's stream.  a owns the twin
// and frees it before its own buffers.
wl_amg *make_twin(wl_amg *a) {
  wl_op *src = a->op;
  wl_op *o = new wl_op();
  o->N = src->N;
  o->m = src->m;
  o->c = src->c;
  o->device = src->device;
  o->geo = src->geo;
  o->gauge_hash = src->gauge_hash;
  o->user = src->stream;
  o->stream = nullptr;
  o->ev = nullptr;
  if (cudaStreamCreateWithFlags(&o->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&o->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    wl_set_error("second solve lane: cannot create a stream or an event");
    if (o->ev) cudaEventDestroy(o->ev);
    if (o->stream) cudaStreamDestroy(o->stream);
    delete o;
    return nullptr;
  }
  o->Uf64 = src->Uf64.view();
  o->Uf32 = src->Uf32.view();
  wl_amg *t = new wl_amg();
  t->op = o;
  t->prm = a->prm;
  t->prm.overlap = 0;
  t->L = a->L;
  for (int l = 0; l < a->L; ++l) {
    const Level &S = a->lev[l];
    Level &D = t->lev[l];
    D.N = S.N;
    D.B = S.B;
    D.n = S.n;
    D.geo = S.geo;
    const LevelOps *so[3] = {&S.op64, &S.op32, &S.opbf};
    LevelOps *dn[3] = {&D.op64, &D.op32, &D.opbf};
    for (int q = 0; q < 3; ++q) {
      dn[q]->A = so[q]->A.view();
      dn[q]->den = so[q]->den.view();
      dn[q]->P = so[q]->P.view();
    }
  }
  t->Ainv = a->Ainv.view();
  t->Ainv32 = a->Ainv32.view();
  t->nc = a->nc;
  t->cap = 0;
  t->cap_prec = a->cap_prec;
  t->h_small = nullptr;
  return t;
}

void amg_free(wl_amg *a) {
  if (!a) return;
  if (a->twin) {  // views a's buffers: goes first
    amg_release(a->twin);
    a->twin = nullptr;
  }
  if (a->op && a->op->stream) cudaStreamSynchronize(a->op->stream);
  release_graphs(a);
  for (int l = 0; l < 8; ++l) {
    Level &L = a->lev[l];
    LevelOps *ops[3] = {&L.op64, &L.op32, &L.opbf};
    for (auto *o : ops) {
      o->A.release();
      o->den.release();
      o->P.release();
    }
    L.x.release();
    L.r.release();
    L.f.release();
    L.t.release();
  }
  a->Ainv.release();
  a->Ainv32.release();
  a->V.release();
  a->Z.release();
  a->w.release();
  a->bh.release();
  a->xh.release();
  a->rr.release();
  a->sb.release();
  a->sx.release();
  a->red.release();
  a->small.release();
  if (a->h_small) cudaFreeHost(a->h_small);
  wl_op *op = a->op;
  delete a;
  if (op) op_release(op);
}

void amg_retain(wl_amg *a) { a->refs.fetch_add(1); }
void amg_release(wl_amg *a) {
  if (a->refs.fetch_sub(1) == 1) amg_free(a);
}

}  // namespace wl

extern "C" void amg_destroy(wl_amg *a) {
  if (a) wl::amg_release(a);
}

extern "C" int amg_levels(wl_amg *a, int *N_out) {
  if (!a) return WL_EINVAL;
  if (N_out)
    for (int l = 0; l < a->L; ++l) N_out[l] = a->lev[l].N;
  return a->L;
}

// ------------------------------------------------------------ file format
extern "C" int amg_export(wl_amg *a, const char *path) {
  if (!a || !path) {
    wl_set_error("amg_export: invalid argument");
    return WL_EINVAL;
  }
  std::vector<unsigned char> buf;
  auto put = [&](const void *p, size_t n) {
    const unsigned char *c = (const unsigned char *)p;
    buf.insert(buf.end(), c, c + n);
  };
  put(kMagic, 8);
  int32_t ver = 1, L = a->L;
  put(&ver, 4);
  put(&L, 4);
  for (int l = 0; l < L; ++l) {
    int32_t v = a->lev[l].N;
    put(&v, 4);
  }
  for (int l = 0; l < L; ++l) {
    int32_t v = a->lev[l].B;
    put(&v, 4);
  }
  WL_TRY(wl::enter(a->op));
  put(&a->op->m, 8);
  put(&a->op->gauge_hash, 8);
  cudaStream_t s = a->op->stream;
  WL_CUDA(cudaStreamSynchronize(s));
  for (int l = 0; l + 1 < L; ++l) {
    std::vector<zd> h((size_t)a->lev[l].n * 8);
    WL_CUDA(cudaMemcpy(h.data(), a->lev[l].op64.P.p, sizeof(zd) * h.size(), cudaMemcpyDeviceToHost));
    put(h.data(), sizeof(zd) * h.size());
  }
  for (int l = 1; l < L; ++l) {
    std::vector<zd> h((size_t)a->lev[l].n * 36);
    WL_CUDA(cudaMemcpy(h.data(), a->lev[l].op64.A.p, sizeof(zd) * h.size(), cudaMemcpyDeviceToHost));
    put(h.data(), sizeof(zd) * h.size());
  }
  uint64_t ck = wl::hash_bytes(buf.data(), buf.size());
  put(&ck, 8);
  FILE *f = fopen(path, "wb");
  if (!f) {
    wl_set_error("amg_export: cannot open %s", path);
    return WL_EINVAL;
  }
  size_t w = fwrite(buf.data(), 1, buf.size(), f);
  fclose(f);
  if (w != buf.size()) {
    wl_set_error("amg_export: short write");
    return WL_EINVAL;
  }
  return WL_OK;
}

extern "C" int amg_import(wl_op *op, const char *path, const amg_params *params, wl_amg **out) {
  if (!op || !path || !out) {
    wl_set_error("amg_import: invalid argument");
    return WL_EINVAL;
  }
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) {
    wl_set_error("amg_import: cannot open %s", path);
    return WL_EINVAL;
  }
  std::vector<unsigned char> buf;
  unsigned char tmp[1 << 16];
  size_t got;
  while ((got = fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
  fclose(f);
  size_t pos = 0;
  auto take = [&](void *p, size_t n) -> bool {
    if (pos + n > buf.size()) return false;
    memcpy(p, buf.data() + pos, n);
    pos += n;
    return true;
  };
  char magic[8];
  int32_t ver = 0, L = 0;
  if (buf.size() < 32 || !take(magic, 8) || memcmp(magic, kMagic, 8) || !take(&ver, 4) || ver != 1 ||
      !take(&L, 4) || L < 2 || L > 8) {
    wl_set_error("amg_import: not a hierarchy file");
    return WL_BAD_HIERARCHY;
  }
  uint64_t ck;
  memcpy(&ck, buf.data() + buf.size() - 8, 8);
  if (wl::hash_bytes(buf.data(), buf.size() - 8) != ck) {
    wl_set_error("amg_import: checksum mismatch");
    return WL_BAD_HIERARCHY;
  }
  int32_t Nl[8], Bl[8];
  double m;
  uint64_t gh;
  for (int l = 0; l < L; ++l)
    if (!take(&Nl[l], 4)) return WL_BAD_HIERARCHY;
  for (int l = 0; l < L; ++l)
    if (!take(&Bl[l], 4)) return WL_BAD_HIERARCHY;
  if (!take(&m, 8) || !take(&gh, 8)) return WL_BAD_HIERARCHY;
  if (Nl[0] != op->N || m != op->m || gh != op->gauge_hash) {
    wl_set_error("amg_import: hierarchy belongs to another operator (N, m or gauge differ)");
    return WL_BAD_HIERARCHY;
  }
  amg_params prm;
  if (params) prm = *params;
  else amg_params_default(&prm);
  prm.levels = L;
  for (int l = 0; l + 1 < L; ++l) prm.block[l] = Bl[l];
  int NN[8];
  int rc = wl::resolve_levels(op->N, &prm, NN);
  if (rc) return WL_BAD_HIERARCHY;
  for (int l = 0; l < L; ++l)
    if (NN[l] != Nl[l]) return WL_BAD_HIERARCHY;
  size_t need = 0;
  for (int l = 0; l + 1 < L; ++l) need += sizeof(zd) * (size_t)Nl[l] * Nl[l] / 2 * 8;
  for (int l = 1; l < L; ++l) need += sizeof(zd) * (size_t)Nl[l] * Nl[l] / 2 * 36;
  if (pos + need + 8 != buf.size()) {
    wl_set_error("amg_import: file size does not match its levels");
    return WL_BAD_HIERARCHY;
  }
  WL_TRY(wl::enter(op));
  wl_amg *a = new wl_amg();
  a->op = op;
  wl::op_retain(op);
  a->prm = prm;
  a->L = L;
  a->cap = 0;
  a->h_small = nullptr;
  rc = wl::hier_alloc(a, Nl);
  cudaStream_t s = op->stream;
  for (int l = 0; l + 1 < L && !rc; ++l) {
    size_t bytes = sizeof(zd) * (size_t)a->lev[l].n * 8;
    if (cudaMemcpy(a->lev[l].op64.P.p, buf.data() + pos, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = WL_ECUDA;
    pos += bytes;
  }
  for (int l = 1; l < L && !rc; ++l) {
    size_t bytes = sizeof(zd) * (size_t)a->lev[l].n * 36;
    if (cudaMemcpy(a->lev[l].op64.A.p, buf.data() + pos, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = WL_ECUDA;
    pos += bytes;
  }
  if (!rc) rc = wl::build_dhat_stencil(op, a->lev[0].op64.A.as<zd>(), s);
  if (!rc) rc = wl::hier_finish(a);
  if (rc) {
    wl::amg_free(a);
    return rc;
  }
  *out = a;
  return WL_OK;
}
