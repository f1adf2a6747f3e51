// wl_serve.cu -- serving runtime: resident hierarchies for several gauge
// fields (lattice sizes may differ) answer a stream of solve requests with
// continuous batching.
//
// Each resident configuration owns a worker thread, its operator's work
// stream and a fixed number of right-hand-side slots sized against the
// server's device-memory budget.  Right-hand sides of queued requests are
// admitted into free slots at every FGMRES restart boundary; the active
// slots are packed into one batch, one restart cycle runs, and slots whose
// true FP64 residual reaches the request's tolerance are retired (their
// solution reconstructed into the request's output) -- so requests that
// arrive while others are on the GPU join as slots free up, and the
// configurations' work overlaps on the device.  A right-hand side's
// arithmetic does not depend on its batch mates (every reduction is per
// right-hand side), so it gets the same result alone and in a mix, up to
// the rounding of the reduction trees.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "wl_common.cuh"

namespace wl {
int fg_norms(wl_amg *a, const zd *v, int nrhs, double *out);
int fg_residual(wl_amg *a, const zd *bh, const zd *xh, int nrhs, double *rnorm);
int fg_cycle(wl_amg *a, const zd *bnorm_h, zd *xh, int nrhs, double tol, const int *active, int *iters_out,
             int *nan_out);
int fg_upload_bnorm(wl_amg *a, const double *bn, int nrhs);
}

// column c of an internal [n2][cap] array <-> column q of a packed [n2][nq]
__global__ void k_pack_cols(const zd *__restrict__ src, int scap, const int *__restrict__ cols, zd *__restrict__ dst,
                            int nq, long n2) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n2 * nq) return;
  long i = tid / nq;
  int q = (int)(tid - i * nq);
  dst[tid] = src[i * scap + cols[q]];
}
__global__ void k_unpack_cols(const zd *__restrict__ src, int nq, const int *__restrict__ cols, zd *__restrict__ dst,
                              int dcap, long n2) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n2 * nq) return;
  long i = tid / nq;
  int q = (int)(tid - i * nq);
  dst[i * dcap + cols[q]] = src[tid];
}
// bhat for one right-hand side into slot column c (stride cap): b_e/c + K_eo b_o/c
__global__ void k_reduce_col(Geo g, double c, const zd *__restrict__ V, const zd *__restrict__ b, zd *bh, int cap,
                             int col) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.nsites()) return;
  int N = g.N, x, y;
  g.xy(h, x, y);
  double ic = 1.0 / c;
  zd o0 = mk(0.0, 0.0), o1 = mk(0.0, 0.0);
  for (int mu = 0; mu < 2; ++mu)
    for (int fwd = 1; fwd >= 0; --fwd) {
      int dx = (mu == 0) ? (fwd ? 1 : -1) : 0, dy = (mu == 1) ? (fwd ? 1 : -1) : 0;
      int xn = (x + dx) & (N - 1), yn = (y + dy) & (N - 1);
      int lx = fwd ? x : xn, ly = fwd ? y : yn;
      zd link = V[(mu * N + ly) * N + lx];
      long j = ((long)yn * N + xn) * 2;
      zd v0 = ic * b[j], v1 = ic * b[j + 1];
      zd w;
      if (mu == 0) w = fwd ? v0 - v1 : v0 + v1;
      else w = fwd ? v0 + ci(v1) : v0 - ci(v1);
      w = (fwd ? link : cconj(link)) * w;
      o0 = o0 + w;
      if (mu == 0) o1 = fwd ? o1 - w : o1 + w;
      else o1 = fwd ? o1 - ci(w) : o1 + ci(w);
    }
  long e = ((long)y * N + x) * 2;
  bh[((long)h * 2) * cap + col] = ic * b[e] + o0;
  bh[((long)h * 2 + 1) * cap + col] = ic * b[e + 1] + o1;
}
// psi for one right-hand side from slot column c: psi_e = x_e, psi_o = b_o/c + K_oe x_e
__global__ void k_reconstruct_col(Geo g, double c, const zd *__restrict__ V, const zd *__restrict__ b,
                                  const zd *__restrict__ xe, int cap, int col, zd *__restrict__ psi) {
  int z = blockIdx.x * blockDim.x + threadIdx.x;
  int N = g.N;
  if (z >= N * N) return;
  int y = z / N, x = z % N;
  if (((x + y) & 1) == 0) {
    long j = (long)g.idx(x, y) * 2 * cap + col;
    psi[(long)z * 2] = xe[j];
    psi[(long)z * 2 + 1] = xe[j + cap];
    return;
  }
  zd o0 = mk(0.0, 0.0), o1 = mk(0.0, 0.0);
  for (int mu = 0; mu < 2; ++mu)
    for (int fwd = 1; fwd >= 0; --fwd) {
      int dx = (mu == 0) ? (fwd ? 1 : -1) : 0, dy = (mu == 1) ? (fwd ? 1 : -1) : 0;
      int xn = (x + dx) & (N - 1), yn = (y + dy) & (N - 1);
      int lx = fwd ? x : xn, ly = fwd ? y : yn;
      zd link = V[(mu * N + ly) * N + lx];
      long j = (long)g.idx(xn, yn) * 2 * cap + col;
      zd v0 = xe[j], v1 = xe[j + cap];
      zd w;
      if (mu == 0) w = fwd ? v0 - v1 : v0 + v1;
      else w = fwd ? v0 + ci(v1) : v0 - ci(v1);
      w = (fwd ? link : cconj(link)) * w;
      o0 = o0 + w;
      if (mu == 0) o1 = fwd ? o1 - w : o1 + w;
      else o1 = fwd ? o1 - ci(w) : o1 + ci(w);
    }
  double ic = 1.0 / c;
  psi[(long)z * 2] = ic * b[(long)z * 2] + o0;
  psi[(long)z * 2 + 1] = ic * b[(long)z * 2 + 1] + o1;
}
__global__ void k_zero_col(zd *v, long n2, int cap, int col) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) v[i * cap + col] = mk(0.0, 0.0);
}

namespace {
using clk = std::chrono::steady_clock;

struct Req {
  long long id;
  int cfg, nrhs, remaining;
  const zd *b;
  zd *x;
  double tol;
  clk::time_point t_arrival, t_done;
  std::vector<wl_info> info;
  bool done = false;
  int status = WL_OK;
};

struct Slot {
  Req *req = nullptr;
  int j = 0;         // right-hand side within the request
  double bnorm = 1;
  int iters = 0, restarts = 0;
};

struct Worker {
  wl_amg *amg;
  int cap;
  DBuf SB, SX, PB, PX, cols;  // slot arrays [n2][cap] and packed arrays [n2][nact]
  std::deque<std::pair<Req *, int>> pending;
  std::vector<Slot> slots;    // size cap; req == nullptr means free
  std::thread th;
  size_t bytes = 0;
};
}  // namespace

struct wl_server {
  size_t budget, used = 0;
  int max_slots;
  std::vector<Worker *> w;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false, started = false;
  long long next_id = 1;
  std::map<long long, Req *> reqs;
  int error = WL_OK;
  std::atomic<long long> solved{0};
};

static void serve_loop(wl_server *S, Worker *W);

extern "C" int srv_create(unsigned long long hbm_budget_bytes, int max_slots_per_config, wl_server **out) {
  if (!out || max_slots_per_config < 1 || max_slots_per_config > 256) {
    wl_set_error("srv_create: 1 <= max_slots_per_config <= 256");
    return WL_EINVAL;
  }
  wl_server *S = new wl_server();
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots_per_config;
  *out = S;
  return WL_OK;
}

// device bytes a configuration needs for `cap` slots (workspace + slot arrays)
static size_t slot_bytes(wl_amg *a, int cap) {
  size_t per = 0;
  for (int l = 0; l < a->L; ++l) per += 4 * sizeof(zd) * (size_t)a->lev[l].n * 2;  // cycle vectors
  size_t n2 = (size_t)a->lev[0].n * 2;
  per += sizeof(zd) * n2 * (2 * a->prm.fgmres_m + 5);  // V, Z, w, bh, xh, rr
  per += sizeof(zd) * n2 * 4;                           // slot and packed arrays
  return per * cap;
}

extern "C" int srv_add(wl_server *S, wl_amg *amg, int *cfg_id) {
  if (!S || !amg || !cfg_id) {
    wl_set_error("srv_add: invalid argument");
    return WL_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->started) {
    wl_set_error("srv_add: the server is already running");
    return WL_EINVAL;
  }
  int cap = S->max_slots;
  size_t need = slot_bytes(amg, cap);
  while (cap > 1 && S->used + need > S->budget) {  // shrink the slot count to the budget
    cap /= 2;
    need = slot_bytes(amg, cap);
  }
  if (S->used + need > S->budget) {
    wl_set_error("srv_add: device-memory budget exhausted (%zu of %zu bytes used, %zu needed)", S->used, S->budget,
                 need);
    return WL_OOM;
  }
  Worker *W = new Worker();
  W->amg = amg;
  W->cap = cap;
  W->slots.resize(cap);
  long n2 = (long)amg->lev[0].n * 2;
  int rc = wl::ensure_workspace(amg, cap, amg->prm.precision);
  if (!rc) rc = W->SB.alloc(sizeof(zd) * n2 * cap);
  if (!rc) rc = W->SX.alloc(sizeof(zd) * n2 * cap);
  if (!rc) rc = W->PB.alloc(sizeof(zd) * n2 * cap);
  if (!rc) rc = W->PX.alloc(sizeof(zd) * n2 * cap);
  if (!rc) rc = W->cols.alloc(sizeof(int) * cap);
  if (rc) {
    W->SB.release();
    W->SX.release();
    W->PB.release();
    W->PX.release();
    W->cols.release();
    delete W;
    return rc;
  }
  W->bytes = need;
  wl::amg_retain(amg);  // the hierarchy outlives the server's use of it
  S->used += need;
  *cfg_id = (int)S->w.size();
  S->w.push_back(W);
  return WL_OK;
}

extern "C" int srv_info(wl_server *S, int cfg, int *slots, unsigned long long *bytes) {
  if (!S || !slots || !bytes) return WL_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (cfg < 0 || cfg >= (int)S->w.size()) {
    wl_set_error("srv_info: no configuration %d", cfg);
    return WL_EINVAL;
  }
  *slots = S->w[cfg]->cap;
  *bytes = S->w[cfg]->bytes;
  return WL_OK;
}

extern "C" int srv_start(wl_server *S) {
  if (!S) return WL_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->started) return WL_OK;
  // capture the cycle graph of every packed width now: a capture while
  // client threads run would make their device-wide synchronisation fail
  for (Worker *W : S->w) {
    wl_amg *a = W->amg;
    WL_CUDA(cudaSetDevice(a->op->device));
    for (int q = 1; q <= W->cap; ++q) WL_TRY(wl::cycle_prepare(a, q, a->prm.precision, a->op->stream, nullptr));
    WL_CUDA(cudaStreamSynchronize(a->op->stream));
  }
  S->started = true;
  for (Worker *W : S->w) W->th = std::thread(serve_loop, S, W);
  return WL_OK;
}

extern "C" int srv_submit(wl_server *S, int cfg, const void *b, void *x, int nrhs, double tol, long long *req_id) {
  if (!S || !b || !x || !req_id || nrhs < 1 || !(tol > 0) || cfg < 0 || cfg >= (int)S->w.size()) {
    wl_set_error("srv_submit: invalid argument");
    return WL_EINVAL;
  }
  Req *R = new Req();
  R->cfg = cfg;
  R->nrhs = nrhs;
  R->remaining = nrhs;
  R->b = (const zd *)b;
  R->x = (zd *)x;
  R->tol = tol;
  R->t_arrival = clk::now();
  R->info.resize(nrhs);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    R->id = S->next_id++;
    S->reqs[R->id] = R;
    for (int j = 0; j < nrhs; ++j) S->w[cfg]->pending.emplace_back(R, j);
    *req_id = R->id;
  }
  S->cv.notify_all();
  return WL_OK;
}

// done = 1 once every right-hand side of the request is solved; latency in
// milliseconds from submission to the retirement of its last right-hand side
extern "C" int srv_poll(wl_server *S, long long req_id, int *done, wl_info *info, double *latency_ms) {
  if (!S || !done) return WL_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->error) return S->error;
  auto it = S->reqs.find(req_id);
  if (it == S->reqs.end()) {
    wl_set_error("srv_poll: unknown request");
    return WL_EINVAL;
  }
  Req *R = it->second;
  *done = R->done ? 1 : 0;
  if (R->done) {
    if (info) memcpy(info, R->info.data(), sizeof(wl_info) * R->nrhs);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(R->t_done - R->t_arrival).count();
    return R->status;
  }
  return WL_OK;
}

// block until every submitted request is done (or an error occurred)
extern "C" int srv_drain(wl_server *S) {
  if (!S) return WL_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv.wait(lk, [&] {
    if (S->error) return true;
    for (auto &kv : S->reqs)
      if (!kv.second->done) return false;
    return true;
  });
  return S->error;
}

extern "C" void srv_destroy(wl_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (Worker *W : S->w) {
    if (W->th.joinable()) W->th.join();
    W->SB.release();
    W->SX.release();
    W->PB.release();
    W->PX.release();
    W->cols.release();
    wl::amg_release(W->amg);
    delete W;
  }
  for (auto &kv : S->reqs) delete kv.second;
  delete S;
}

static int worker_step(wl_server *S, Worker *W) {
  wl_amg *a = W->amg;
  wl_op *op = a->op;
  cudaStream_t s = op->stream;
  long n2 = (long)a->lev[0].n * 2;
  int cap = W->cap;
  // admit queued right-hand sides into free slots
  std::vector<std::pair<Req *, int>> admit;
  std::vector<int> admit_col;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (int c = 0; c < cap && !W->pending.empty(); ++c)
      if (!W->slots[c].req) {
        admit.push_back(W->pending.front());
        admit_col.push_back(c);
        W->slots[c].req = W->pending.front().first;  // reserve
        W->pending.pop_front();
      }
  }
  for (size_t q = 0; q < admit.size(); ++q) {
    Req *R = admit[q].first;
    int j = admit[q].second, c = admit_col[q];
    const zd *bj = R->b + (size_t)j * op->N * op->N * 2;
    k_reduce_col<<<WL_GRID(a->lev[0].n, 128), 128, 0, s>>>(op->geo, op->c, op->Uf64.as<zd>(), bj, W->SB.as<zd>(),
                                                            cap, c);
    k_zero_col<<<WL_GRID(n2, 256), 256, 0, s>>>(W->SX.as<zd>(), n2, cap, c);
    wl_count_launches(2);
    Slot &sl = W->slots[c];
    sl.req = R;
    sl.j = j;
    sl.iters = 0;
    sl.restarts = 0;
    sl.bnorm = -1;  // computed below
  }
  // pack the active slots
  std::vector<int> cols;
  for (int c = 0; c < cap; ++c)
    if (W->slots[c].req) cols.push_back(c);
  int nq = (int)cols.size();
  if (nq == 0) return 0;
  WL_CUDA(cudaMemcpyAsync(W->cols.p, cols.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
  k_pack_cols<<<WL_GRID(n2 * nq, 256), 256, 0, s>>>(W->SB.as<zd>(), cap, W->cols.as<int>(), W->PB.as<zd>(), nq, n2);
  k_pack_cols<<<WL_GRID(n2 * nq, 256), 256, 0, s>>>(W->SX.as<zd>(), cap, W->cols.as<int>(), W->PX.as<zd>(), nq, n2);
  wl_count_launches(2);
  std::vector<double> bn(nq), rn(nq);
  bool need_bn = false;
  for (int q = 0; q < nq; ++q) need_bn |= W->slots[cols[q]].bnorm < 0;
  if (need_bn) {
    WL_TRY(wl::fg_norms(a, W->PB.as<zd>(), nq, bn.data()));
    for (int q = 0; q < nq; ++q)
      if (W->slots[cols[q]].bnorm < 0) W->slots[cols[q]].bnorm = bn[q] > 0 ? bn[q] : 1.0;
  }
  for (int q = 0; q < nq; ++q) bn[q] = W->slots[cols[q]].bnorm;
  WL_TRY(wl::fg_residual(a, W->PB.as<zd>(), W->PX.as<zd>(), nq, rn.data()));
  // retire converged slots (reconstruct psi into the request's output)
  std::vector<int> active(nq, 0);
  int nact = 0;
  for (int q = 0; q < nq; ++q) {
    Slot &sl = W->slots[cols[q]];
    double rel = rn[q] / sl.bnorm;
    bool bad = !std::isfinite(rel);  // retired alone; the other slots go on
    bool conv = !bad && rel <= sl.req->tol;
    bool give_up = bad || sl.restarts >= a->prm.max_restarts;
    if (conv || give_up) {
      Req *R = sl.req;
      const zd *bj = R->b + (size_t)sl.j * op->N * op->N * 2;
      zd *xj = R->x + (size_t)sl.j * op->N * op->N * 2;
      k_reconstruct_col<<<WL_GRID(op->N * op->N, 256), 256, 0, s>>>(op->geo, op->c, op->Uf64.as<zd>(), bj,
                                                                    W->SX.as<zd>(), cap, cols[q], xj);
      wl_count_launches(1);
      WL_CUDA(cudaStreamSynchronize(s));
      std::lock_guard<std::mutex> lk(S->mu);
      wl_info &inf = R->info[sl.j];
      inf.status = bad ? WL_NAN : conv ? WL_OK : WL_NOT_CONVERGED;
      inf.iters = sl.iters;
      inf.restarts = sl.restarts;
      inf.true_relres = rel;
      if (bad) R->status = WL_NAN;
      else if (!conv && R->status != WL_NAN) R->status = WL_NOT_CONVERGED;
      if (--R->remaining == 0) {
        R->t_done = clk::now();
        R->done = true;
        S->cv.notify_all();
      }
      S->solved++;
      sl.req = nullptr;
    } else {
      active[q] = 1;
      nact++;
    }
  }
  if (nact == 0) return 1;
  // one restart cycle on the packed batch (retired columns are inactive);
  // inside the cycle the smallest requested tolerance decides when an
  // Arnoldi process stops, each request's own tolerance decides retirement
  WL_TRY(wl::fg_upload_bnorm(a, bn.data(), nq));
  std::vector<int> it(nq, 0);
  double tol = 1.0;
  for (int q = 0; q < nq; ++q)
    if (active[q]) tol = std::min(tol, W->slots[cols[q]].req->tol);
  WL_TRY(wl::fg_cycle(a, nullptr, W->PX.as<zd>(), nq, tol, active.data(), it.data(), nullptr));
  for (int q = 0; q < nq; ++q)
    if (active[q]) {
      W->slots[cols[q]].iters += it[q];
      W->slots[cols[q]].restarts++;
    }
  k_unpack_cols<<<WL_GRID(n2 * nq, 256), 256, 0, s>>>(W->PX.as<zd>(), nq, W->cols.as<int>(), W->SX.as<zd>(), cap, n2);
  wl_count_launches(1);
  WL_CUDA(cudaGetLastError());
  return 1;
}

static void serve_loop(wl_server *S, Worker *W) {
  cudaSetDevice(W->amg->op->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        if (S->stop || S->error) return true;
        if (!W->pending.empty()) return true;
        for (auto &sl : W->slots)
          if (sl.req) return true;
        return false;
      });
      if (S->stop || S->error) return;
    }
    int rc = worker_step(S, W);
    if (rc < 0) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->error = rc;
      S->cv.notify_all();
      return;
    }
  }
}
