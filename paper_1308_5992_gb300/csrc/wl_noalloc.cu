// wl_noalloc.cu -- y = Dhat x without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need this
// operator: a process whose device memory is already reserved by its own pool
// (for example a framework's caching allocator holding most of the HBM, so a
// raw cudaMalloc fails), or a latency-critical loop that cannot accept the
// device-wide synchronisation that cudaMalloc / cudaFree imply.  For them,
// wl_dhat_apply_noalloc keeps the odd-site intermediate K_oe x of the two-hop
// product in a fixed, file-scope device array instead of a buffer it would
// have to allocate.  The array holds WL_NOALLOC_MAX_COMPLEX complex doubles
// (16 MiB) on every GPU that loads this library, for the life of the process.
//
// The array's name in host code is only a host-side stand-in: its device
// address is fetched with cudaGetSymbolAddress once per device (with that
// device current) by the first call on that device and cached for the life
// of the process, so the library must not be used across a cudaDeviceReset
// (the cached address would be stale).  The call synchronises its stream
// before returning, so it must not be issued during a stream capture.  Every call
// shares the array: the first kernel overwrites every element it later reads,
// so nothing needs clearing, but two calls whose work overlaps on the GPU
// (on different streams or operators) race on it.
#include <mutex>

#include "wl_common.cuh"

#define WL_NOALLOC_MAX_COMPLEX (1 << 20)
#define WL_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) zd g_noalloc_odd[WL_NOALLOC_MAX_COMPLEX];

static std::mutex g_noalloc_mu;
static zd *g_noalloc_ptr[WL_NOALLOC_MAX_DEVICES];

// device address of the scratch array on device `dev`, which must be the
// current device (set up once per device)
static int noalloc_scratch(int dev, zd **out) {
  if (dev < 0 || dev >= WL_NOALLOC_MAX_DEVICES) {
    wl_set_error("wl_dhat_apply_noalloc: device %d out of range", dev);
    return WL_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_odd);
    if (e != cudaSuccess || !p) {
      wl_set_error("wl_dhat_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return WL_ECUDA;
    }
    g_noalloc_ptr[dev] = (zd *)p;
  }
  *out = g_noalloc_ptr[dev];
  return WL_OK;
}

// one hop sum on the caller's layout [nrhs][n][2]: out(h) = (sub(h) -) sum of
// the four hops K applied to `in` at the neighbours of h (other parity)
__global__ void k_hop_noalloc(Geo g, const zd *__restrict__ V, int par_out, const zd *__restrict__ in,
                              const zd *__restrict__ sub, zd *__restrict__ out, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int n = g.nsites(), N = g.N;
  if (tid >= (long)n * nrhs) return;
  int r = (int)(tid / n), h = (int)(tid - (long)r * n);
  int y = h >> (g.lg - 1);
  int x = ((h & (g.half() - 1)) << 1) | ((y + par_out) & 1);
  const zd *inr = in + (long)r * n * 2;
  zd o0 = mk(0.0, 0.0), o1 = mk(0.0, 0.0);
  for (int mu = 0; mu < 2; ++mu)
    for (int fwd = 1; fwd >= 0; --fwd) {
      int dx = (mu == 0) ? (fwd ? 1 : -1) : 0, dy = (mu == 1) ? (fwd ? 1 : -1) : 0;
      int xn = (x + dx) & (N - 1), yn = (y + dy) & (N - 1);
      int lx = fwd ? x : xn, ly = fwd ? y : yn;
      zd link = V[(mu * N + ly) * N + lx];
      long j = (long)g.idx(xn, yn) * 2;
      zd v0 = inr[j], v1 = inr[j + 1];
      zd w;
      if (mu == 0) w = fwd ? v0 - v1 : v0 + v1;
      else w = fwd ? v0 + ci(v1) : v0 - ci(v1);
      w = (fwd ? link : cconj(link)) * w;
      o0 = o0 + w;
      if (mu == 0) o1 = fwd ? o1 - w : o1 + w;
      else o1 = fwd ? o1 - ci(w) : o1 + ci(w);
    }
  long o = ((long)r * n + h) * 2;
  if (sub) {
    o0 = sub[o] - o0;
    o1 = sub[o + 1] - o1;
  }
  out[o] = o0;
  out[o + 1] = o1;
}

extern "C" int wl_dhat_apply_noalloc(wl_op *op, const void *x, void *y, int nrhs) {
  if (!op || !x || !y || nrhs < 1) {
    wl_set_error("wl_dhat_apply_noalloc: invalid argument");
    return WL_EINVAL;
  }
  long n = op->geo.nsites();
  if (n * 2 * (long)nrhs > WL_NOALLOC_MAX_COMPLEX) {
    wl_set_error("wl_dhat_apply_noalloc: %ld complex values of scratch needed (L = %d, nrhs = %d), the fixed "
                 "array holds %d; use wl_apply",
                 n * 2 * (long)nrhs, op->N, nrhs, WL_NOALLOC_MAX_COMPLEX);
    return WL_EINVAL;
  }
  int prev = 0;
  WL_CUDA(cudaGetDevice(&prev));
  if (prev != op->device) WL_CUDA(cudaSetDevice(op->device));
  zd *t = nullptr;
  int rc = noalloc_scratch(op->device, &t);
  if (!rc) rc = wl::enter(op);
  if (rc) {
    if (prev != op->device) cudaSetDevice(prev);
    return rc;
  }
  cudaStream_t s = op->stream;
  unsigned grid = WL_GRID(n * nrhs, 256);
  k_hop_noalloc<<<grid, 256, 0, s>>>(op->geo, op->Uf64.as<zd>(), 1, (const zd *)x, nullptr, t, nrhs);
  k_hop_noalloc<<<grid, 256, 0, s>>>(op->geo, op->Uf64.as<zd>(), 0, t, (const zd *)x, (zd *)y, nrhs);
  wl_count_launches(2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (prev != op->device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    wl_set_error("wl_dhat_apply_noalloc: %s", cudaGetErrorString(e));
    return WL_ECUDA;
  }
  return WL_OK;
}
