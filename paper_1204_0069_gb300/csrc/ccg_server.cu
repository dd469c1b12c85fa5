// ccg_server.cu -- serving loop for streams of SPD solve requests
// (include/ccg.h, "Serving").  Host code: a pool of worker threads, each with
// its own solver handle, stream and fixed share of the SMs; a shared queue
// from which a free worker admits the oldest request that fits the remaining
// device-memory budget (first fit in arrival order); per-request timestamps.
// Requests admitted while others run execute concurrently on the device.  A
// request's grid depends only on its size and the worker share, so its result
// is the same whether it runs alone or in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ccg.h"
#include "ccg_handle.h"
#include "ccg_internal.h"

using namespace ccg_host;

namespace {

struct Request {
  int64_t id;
  int64_t n, lda;
  const double* A;
  const double* b;
  double* x;
  int p;
  double tol;
  int maxit;
  double reserve;
  double t_submit;
};

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct ccg_server_s {
  ccg_server_config cfg;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work;
  std::condition_variable cv_done;
  std::deque<Request> pending;
  std::deque<ccg_server_result> done;
  double reserved = 0.0;
  double peak_reserved = 0.0;
  int in_flight = 0;
  int peak_in_flight = 0;
  int64_t completed = 0;
  bool stop = false;
  int shares = 0;
  std::vector<std::thread> workers;
  std::vector<ccg_handle*> handles;
  std::vector<cudaStream_t> streams;
};

namespace {

// Device bytes a request holds while it runs: its matrix (resident for the
// request's lifetime), the quantised copy of the mixed-precision path (and,
// for BF16 / FP8, the sliced copy of the preconditioned FP64 solve), and the
// solver workspace (blocks, partial sums, operand rows, partial tiles).
double reservation(const ccg_server_config& c, int64_t n, int64_t lda, int p, int shares) {
  const double a = (double)n * (double)lda * 8.0;
  const double ld = (double)((n + 127) / 128 * 128);
  double lp = 0.0;
  if (c.precision == CCG_FP32_IR) lp = (double)n * ld * 4.0 + 64.0 * ld * 4.0;
  else if (c.precision == CCG_BF16_IR) lp = (double)n * ld * 2.0 + 32.0 * ld * 2.0;
  else if (c.precision == CCG_FP8_IR) lp = (double)n * ld * 1.0 + 64.0 * ld + 4.0 * n;
  const double sliced =
      14.0 * ld * ld + 4.0 * n + 224.0 * ld + (shares + ld / 128.0) * 128.0 * p * 8.0;
  if (c.precision == CCG_FP64_SLICED)  // 14 slices, operand slices, FP64 partial tiles
    lp = sliced;
  else if (c.precision == CCG_BF16_IR || c.precision == CCG_FP8_IR)
    // the preconditioned FP64 solve (the default method for BF16 / FP8) also
    // holds the sliced copy and four more n x p blocks
    lp += (p <= 16 ? sliced : 0.0) + 4.0 * n * p * 8.0;
  const double ws = 5.0 * n * p * 8.0 + shares * ccg::kPartStride * 8.0 + 6.0 * n * 8.0 +
                    (double)(shares + (n + 127) / 128) * 128.0 * 32.0 * 4.0 + 65536.0;
  return a + lp + ws;
}

void worker_main(ccg_server_s* s, int k) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    Request r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop && s->pending.empty()) return;
        auto it = std::find_if(s->pending.begin(), s->pending.end(), [&](const Request& q) {
          return s->reserved + q.reserve <= s->cfg.budget_bytes;
        });
        if (it != s->pending.end()) {
          r = *it;
          s->pending.erase(it);
          s->reserved += r.reserve;
          s->peak_reserved = std::max(s->peak_reserved, s->reserved);
          ++s->in_flight;
          s->peak_in_flight = std::max(s->peak_in_flight, s->in_flight);
          break;
        }
        s->cv_work.wait(lk);
      }
    }
    const double t_admit = now_ms(s->t0);
    ccg_result res;
    const int st = ccg_solve(s->handles[k], r.n, r.A, r.lda, r.b, nullptr, r.p, r.tol, r.maxit,
                             r.x, &res);
    const double t_done = now_ms(s->t0);
    ccg_server_result out;
    std::memset(&out, 0, sizeof(out));
    out.id = r.id;
    out.status = st;
    out.iterations = res.iterations;
    out.outer_steps = res.outer_steps;
    out.relres_true = res.relres_true;
    out.submit_ms = r.t_submit;
    out.admit_ms = t_admit;
    out.done_ms = t_done;
    out.worker = k;
    out.ctas = res.ctas;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->reserved -= r.reserve;
      --s->in_flight;
      ++s->completed;
      s->done.push_back(out);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

void ccg_server_config_init(ccg_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->device = 0;
  c->workers = 8;
  c->precision = CCG_FP64;
  c->budget_bytes = 150e9;
  c->ctas_per_worker = 0;
}

int ccg_server_create(const ccg_server_config* cfg, ccg_server** out) {
  if (!out) return CCG_ERR_INVALID;
  *out = nullptr;
  ccg_server_config c;
  if (cfg) c = *cfg;
  else ccg_server_config_init(&c);
  if (c.workers < 1 || c.workers > 64 || !(c.budget_bytes > 0.0) || c.ctas_per_worker < 0)
    return CCG_ERR_INVALID;
  int sms = 0;
  if (cudaSetDevice(c.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess) {
    cudaGetLastError();
    return CCG_ERR_INVALID;
  }
  ccg_server_s* s = new (std::nothrow) ccg_server_s();
  if (!s) return CCG_ERR_OOM;
  s->cfg = c;
  s->t0 = std::chrono::steady_clock::now();
  // fixed SM share per worker: concurrent persistent solves stay co-resident
  s->shares = c.ctas_per_worker > 0 ? c.ctas_per_worker : std::max(1, sms / c.workers);
  for (int k = 0; k < c.workers; ++k) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      ccg_server_destroy(s);
      return CCG_ERR_CUDA;
    }
    s->streams.push_back(st);
    ccg_config hc;
    ccg_config_init(&hc);
    hc.device = c.device;
    hc.stream = st;
    hc.precision = c.precision;
    hc.max_ctas = s->shares;
    ccg_handle* h = nullptr;
    const int rc = ccg_create(&h, &hc);
    if (rc != CCG_OK) {
      ccg_server_destroy(s);
      return rc;
    }
    s->handles.push_back(h);
  }
  for (int k = 0; k < c.workers; ++k) s->workers.emplace_back(worker_main, s, k);
  *out = s;
  return CCG_OK;
}

int ccg_server_submit(ccg_server* s, int64_t id, int64_t n, const double* A, int64_t lda,
                      const double* b, double* x_out, int p, double tol, int maxit) {
  if (!s || n < 1 || lda < n || p < 1 || p > ccg::kMaxP || p > n || !(tol > 0.0) || maxit < 0 ||
      !A || !b || !x_out)
    return CCG_ERR_INVALID;
  Request r;
  r.id = id;
  r.n = n;
  r.lda = lda;
  r.A = A;
  r.b = b;
  r.x = x_out;
  r.p = p;
  r.tol = tol;
  r.maxit = maxit;
  r.reserve = reservation(s->cfg, n, lda, p, s->shares);
  if (r.reserve > s->cfg.budget_bytes) return CCG_ERR_OOM;  // can never be admitted
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return CCG_ERR_INVALID;
    r.t_submit = now_ms(s->t0);
    s->pending.push_back(r);
  }
  s->cv_work.notify_one();
  return CCG_OK;
}

int ccg_server_poll(ccg_server* s, ccg_server_result* out, int max, int wait_ms) {
  if (!s || !out || max < 1) return CCG_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  int k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  return k;
}

int ccg_server_stats(ccg_server* s, ccg_server_stats_t* st) {
  if (!s || !st) return CCG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  st->queued = (int64_t)s->pending.size();
  st->in_flight = s->in_flight;
  st->peak_in_flight = s->peak_in_flight;
  st->completed = s->completed;
  st->reserved_bytes = s->reserved;
  st->peak_reserved_bytes = s->peak_reserved;
  st->ctas_per_worker = s->shares;
  st->now_ms = now_ms(s->t0);
  return CCG_OK;
}

int ccg_server_destroy(ccg_server* s) {
  if (!s) return CCG_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  for (ccg_handle* h : s->handles) ccg_destroy(h);
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete s;
  return CCG_OK;
}

}  // extern "C"
