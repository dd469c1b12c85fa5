// ccg_server.cu -- serving loop for streams of SPD solve requests
// (include/ccg.h, "Serving").  Host code only.
//
// Worker mode: a pool of worker threads, each with its own solver handle,
// stream and fixed share of the SMs; a shared queue from which a free worker
// admits the oldest request that fits the remaining device-memory budget
// (first fit in arrival order); per-request timestamps.  Requests admitted
// while others run execute concurrently on the device.
//
// Slots mode: one persistent serving kernel (serve_kernel, ccg_solver.cuh)
// whose slots of CTAs take requests from a ring in mapped host memory.  A
// dispatcher thread admits requests into the ring (first fit under the
// budget), watches the ring entries' claim and completion words, and
// launches the kernel again when it has ended on idle and requests wait.
//
// A request's grid depends only on its size and the worker share (or slot
// size), so its result is the same whether it runs alone or in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
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

// Slots mode: the serving kernel's resources and the ring bookkeeping.
struct SlotMode {
  int slots = 0, group = 0, P = 0, capacity = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_end = nullptr;
  bool launched = false;
  // device memory: slot workspace, partial slots, states, slot barriers, claim counter
  double* ws = nullptr;
  double* part = nullptr;
  ccg::DevState* st = nullptr;
  ccg::SlotSync* sync = nullptr;
  ccg::ServeCtl* ctl = nullptr;
  int64_t ws_stride = 0;
  double fixed_bytes = 0.0;  // slot workspace and partial slots
  // mapped host memory: request ring, its tail and stop words, results
  ccg::ServeDesc* desc = nullptr;
  int* tail = nullptr;
  int* stop = nullptr;
  ccg::ServeOut* out = nullptr;
  // ring entries: posted so far, the request of each entry, open entries
  int posted = 0;
  std::vector<Request> req;
  std::vector<char> open, seen_claim;
  std::vector<double> t_claim;
  std::thread dispatcher;
};

struct ccg_server_s {
  ccg_server_config cfg;
  SlotMode sm;
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
  bool failed = false;  // slots mode: a launch failed; open requests report CCG_ERR_CUDA
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

// ---- slots mode ---------------------------------------------------------

int64_t load_acquire(const int64_t* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

// Launch the serving kernel once more (it ended on idle, or never ran).
cudaError_t launch_slots(ccg_server_s* s) {
  SlotMode& m = s->sm;
  ccg::ServeCtl c;
  std::memset(&c, 0, sizeof(c));
  // the claim counter keeps counting across launches
  cudaError_t e = cudaMemcpyAsync(&c.head, &m.ctl->head, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                  m.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m.ctl, &c, sizeof(c), cudaMemcpyHostToDevice, m.stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(m.sync, 0, sizeof(ccg::SlotSync) * m.slots, m.stream);
  ccg::Params prm{};
  prm.spread = 1.0;
  prm.seed = 0;
  prm.X = m.ws;
  prm.part = m.part;
  prm.st = m.st;
  prm.p = 1;
  prm.rank_tol = 1e-12;
  prm.replacement = 1;
  prm.mode = ccg::MODE_SOLVE;
  prm.timeout_ns = 10000LL * 1000000LL;
  prm.serve_group = m.group;
  prm.serve_capacity = m.capacity;
  ccg::ServeDesc* d_desc = nullptr;
  int *d_tail = nullptr, *d_stop = nullptr;
  ccg::ServeOut* d_out = nullptr;
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_desc), m.desc, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_tail), m.tail, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_stop), m.stop, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_out), m.out, 0);
  prm.serve_desc = d_desc;
  prm.serve_tail = d_tail;
  prm.serve_stop = d_stop;
  prm.serve_out = d_out;
  prm.serve_sync = m.sync;
  prm.serve_ctl = m.ctl;
  prm.serve_ws_stride = m.ws_stride;
  prm.serve_idle_ns = 20LL * 1000000LL;
  if (e == cudaSuccess) e = ccg::launch_serve(prm, m.P, m.slots * m.group, m.stream);
  if (e == cudaSuccess) e = cudaEventRecord(m.ev_end, m.stream);
  m.launched = e == cudaSuccess;
  return e;
}

// Dispatcher of slots mode: completions, admissions, launches.
void dispatcher_main(ccg_server_s* s) {
  cudaSetDevice(s->cfg.device);
  SlotMode& m = s->sm;
  int64_t oldest = 0;  // ring position of the oldest entry not yet done
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    const double now = now_ms(s->t0);
    // completions and claims (entries finish out of order)
    int running = 0;
    bool unclaimed = false;
    for (int64_t pos = oldest; pos < m.posted; ++pos) {
      const int k = (int)(pos % m.capacity);
      if (!m.open[k]) continue;
      const ccg::ServeOut& o = m.out[k];
      if (load_acquire(&o.done) == pos + 1) {
        const Request& r = m.req[k];
        ccg_server_result res;
        std::memset(&res, 0, sizeof(res));
        res.id = r.id;
        res.status = o.status;
        res.iterations = o.iterations;
        res.relres_true = o.relres_true;
        res.worker = o.slot;
        res.ctas = m.group;
        res.submit_ms = r.t_submit;
        res.admit_ms = m.seen_claim[k] ? m.t_claim[k] : now;
        res.done_ms = now;
        s->done.push_back(res);
        s->reserved -= r.reserve;
        ++s->completed;
        --s->in_flight;
        m.open[k] = 0;
        s->cv_done.notify_all();
      } else if (load_acquire(&o.claimed) == pos + 1) {
        if (!m.seen_claim[k]) {
          m.seen_claim[k] = 1;
          m.t_claim[k] = now;
        }
        ++running;
      } else {
        unclaimed = true;
      }
    }
    while (oldest < m.posted && !m.open[oldest % m.capacity]) ++oldest;
    s->peak_in_flight = std::max(s->peak_in_flight, running);
    // admission: first fit in arrival order, while the ring has room
    for (auto it = s->pending.begin();
         it != s->pending.end() && m.posted - oldest < m.capacity;) {
      if (s->reserved + it->reserve > s->cfg.budget_bytes) {
        ++it;
        continue;
      }
      const int pos = m.posted;
      const int k = pos % m.capacity;
      ccg::ServeDesc& d = m.desc[k];
      d.n = it->n;
      d.lda = it->lda;
      d.A = it->A;
      d.b = it->b;
      d.x = it->x;
      d.tol = it->tol;
      d.maxit = it->maxit;
      d.p = it->p;
      __atomic_store_n(&d.seq, (int64_t)pos + 1, __ATOMIC_RELEASE);
      m.req[k] = *it;
      m.open[k] = 1;
      m.seen_claim[k] = 0;
      s->reserved += it->reserve;
      s->peak_reserved = std::max(s->peak_reserved, s->reserved);
      ++s->in_flight;
      m.posted = pos + 1;
      __atomic_store_n(m.tail, m.posted, __ATOMIC_RELEASE);
      unclaimed = true;
      it = s->pending.erase(it);
    }
    // the kernel ends when idle; launch it again while requests wait
    const bool ended = !m.launched || cudaEventQuery(m.ev_end) == cudaSuccess;
    if (ended && unclaimed && !s->failed) {
      if (launch_slots(s) != cudaSuccess) s->failed = true;
    }
    if (s->failed) {
      // report every open request as failed and give up
      for (int64_t pos = oldest; pos < m.posted; ++pos) {
        const int k = (int)(pos % m.capacity);
        if (!m.open[k]) continue;
        ccg_server_result res;
        std::memset(&res, 0, sizeof(res));
        res.id = m.req[k].id;
        res.status = CCG_ERR_CUDA;
        res.submit_ms = m.req[k].t_submit;
        res.done_ms = now;
        s->done.push_back(res);
        m.open[k] = 0;
        --s->in_flight;
        s->reserved -= m.req[k].reserve;
      }
      oldest = m.posted;
      s->cv_done.notify_all();
    }
    if (s->stop && s->pending.empty() && oldest == m.posted) {
      // nothing left: let the kernel leave and wait for it
      __atomic_store_n(m.stop, 1, __ATOMIC_RELEASE);
      lk.unlock();
      if (m.launched) cudaEventSynchronize(m.ev_end);
      return;
    }
    s->cv_work.wait_for(lk, std::chrono::microseconds(50));
  }
}

// Slots mode: resources of the serving kernel and the dispatcher thread.
int create_slots(ccg_server_s* s, int sms) {
  SlotMode& m = s->sm;
  ccg_server_config& c = s->cfg;
  if (c.max_n == 0) c.max_n = 16384;
  if (c.max_p == 0) c.max_p = 8;
  m.slots = c.slots;
  m.group = sms / c.slots;
  m.P = c.max_p <= 8 ? 8 : 32;
  m.capacity = 4096;
  s->shares = m.group;
  if (ccg::serve_ctas_per_sm(m.P) < 1) return CCG_ERR_CUDA;
  m.ws_stride = 5 * c.max_n * (int64_t)m.P;
  const size_t ws_bytes = (size_t)m.slots * m.ws_stride * sizeof(double);
  const size_t part_bytes = (size_t)m.slots * m.group * ccg::kPartStride * sizeof(double);
  cudaError_t e = cudaStreamCreateWithFlags(&m.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m.ev_end, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&m.ws), ws_bytes);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&m.part), part_bytes);
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&m.st), sizeof(ccg::DevState) * m.slots);
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&m.sync), sizeof(ccg::SlotSync) * m.slots);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&m.ctl), sizeof(ccg::ServeCtl));
  if (e == cudaSuccess) e = cudaMemset(m.st, 0, sizeof(ccg::DevState) * m.slots);
  if (e == cudaSuccess) e = cudaMemset(m.ctl, 0, sizeof(ccg::ServeCtl));
  const unsigned fl = cudaHostAllocMapped | cudaHostAllocPortable;
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&m.desc), sizeof(ccg::ServeDesc) * m.capacity, fl);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&m.out), sizeof(ccg::ServeOut) * m.capacity, fl);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&m.tail), 2 * sizeof(int), fl);
  if (e != cudaSuccess) return map_cuda(e);
  m.stop = m.tail + 1;
  std::memset(m.desc, 0, sizeof(ccg::ServeDesc) * m.capacity);
  std::memset(m.out, 0, sizeof(ccg::ServeOut) * m.capacity);
  m.tail[0] = 0;
  m.tail[1] = 0;
  m.req.resize(m.capacity);
  m.open.assign(m.capacity, 0);
  m.seen_claim.assign(m.capacity, 0);
  m.t_claim.assign(m.capacity, 0.0);
  // the slots' blocks are held for the server's life
  m.fixed_bytes = (double)(ws_bytes + part_bytes);
  s->reserved = m.fixed_bytes;
  s->peak_reserved = s->reserved;
  if (s->reserved > c.budget_bytes) return CCG_ERR_OOM;
  m.dispatcher = std::thread(dispatcher_main, s);
  return CCG_OK;
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
  c->slots = 0;
  c->max_n = 16384;
  c->max_p = 8;
}

int ccg_server_create(const ccg_server_config* cfg, ccg_server** out) {
  if (!out) return CCG_ERR_INVALID;
  *out = nullptr;
  ccg_server_config c;
  if (cfg) c = *cfg;
  else ccg_server_config_init(&c);
  // everything that does not depend on the device is checked before the
  // first CUDA call
  if (c.workers < 1 || c.workers > 64 || !(c.budget_bytes > 0.0) || c.ctas_per_worker < 0 ||
      (c.precision != CCG_FP64 && c.precision != CCG_FP32_IR && c.precision != CCG_BF16_IR &&
       c.precision != CCG_FP8_IR && c.precision != CCG_FP64_SLICED) ||
      c.slots < 0 || c.max_n < 0 || c.max_p < 0 || c.max_p > ccg::kMaxP ||
      (c.slots > 0 && c.precision != CCG_FP64))
    return CCG_ERR_INVALID;
  int sms = 0;
  if (cudaSetDevice(c.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess) {
    cudaGetLastError();
    return CCG_ERR_INVALID;
  }
  if (c.slots > sms) return CCG_ERR_INVALID;
  ccg_server_s* s = new (std::nothrow) ccg_server_s();
  if (!s) return CCG_ERR_OOM;
  s->cfg = c;
  s->t0 = std::chrono::steady_clock::now();
  if (c.slots > 0) {
    const int rc = create_slots(s, sms);
    if (rc != CCG_OK) {
      ccg_server_destroy(s);
      return rc;
    }
    *out = s;
    return CCG_OK;
  }
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
  if (s->cfg.slots > 0) {
    // the serving kernel reads A, b and x in place with 16-byte loads of A
    if (n > s->cfg.max_n || p > s->cfg.max_p || (lda & 1) || !aligned(A, 16) ||
        !aligned(b, 8) || !aligned(x_out, 8) || !is_device_ptr(A) || !is_device_ptr(b) ||
        !is_device_ptr(x_out))
      return CCG_ERR_INVALID;
    r.reserve = (double)n * (double)lda * 8.0;
    // the slots' own blocks stay reserved for the server's life
    if (r.reserve + s->sm.fixed_bytes > s->cfg.budget_bytes) return CCG_ERR_OOM;
  } else {
    r.reserve = reservation(s->cfg, n, lda, p, s->shares);
  }
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
  SlotMode& m = s->sm;
  if (m.dispatcher.joinable()) m.dispatcher.join();
  if (m.stream) cudaStreamSynchronize(m.stream);
  if (m.ws) cudaFree(m.ws);
  if (m.part) cudaFree(m.part);
  if (m.st) cudaFree(m.st);
  if (m.sync) cudaFree(m.sync);
  if (m.ctl) cudaFree(m.ctl);
  if (m.desc) cudaFreeHost(m.desc);
  if (m.out) cudaFreeHost(m.out);
  if (m.tail) cudaFreeHost(m.tail);
  if (m.ev_end) cudaEventDestroy(m.ev_end);
  if (m.stream) cudaStreamDestroy(m.stream);
  delete s;
  return CCG_OK;
}

}  // extern "C"
