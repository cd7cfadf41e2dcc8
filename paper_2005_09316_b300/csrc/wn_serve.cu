// Continuous-batching request server for predict / peel requests of uneven size.
//
// A scheduler thread owns the GPU side:
//  * admission by memory: each request's output visibilities are carved from one device pool
//    (first fit); a request waits until a slot (max_inflight) and pool space are free, and one that
//    can never fit is refused at submit (WN_EBUSY);
//  * batching: all admitted requests that are not yet running are packed into one work table of
//    (request, row tile, channel block) entries and run by the persistent batched phasor kernel,
//    replayed from a CUDA graph captured once per stream; shapelet components follow per request on
//    the same stream, with that stream's own tables;
//  * overlap: there are n_streams batch slots; requests that arrive while batches are on the GPU are
//    admitted as memory and slots free up and go out in the next batch on a free stream, so their
//    work overlaps the batches in flight;
//  * completion: an event per batch, polled without blocking; the caller reads the result in place
//    and releases it, which returns its pool space.
// Every tile is computed by the same code in the same order as a single-request launch, so a request's
// result does not depend on what it was batched with.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "wn_internal.cuh"

namespace wn {

enum ReqState { RQ_PENDING = 0, RQ_ADMITTED = 1, RQ_RUNNING = 2, RQ_DONE = 3, RQ_CANCELLED = 4, RQ_FAILED = 5 };

struct ServeReq {
  uint64_t ticket = 0;
  ObsDev od;
  const Model* M = nullptr;
  int mode = OUT_STORE;
  PeelArgs pa;
  size_t bytes = 0, off = 0;
  bool has_mem = false;
  int state = RQ_PENDING;
  int batch = -1;
  int error = WN_OK;
  double t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
};

struct ServeSlot {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t gexec = nullptr;
  char* d_table = nullptr;  // [n_work int (16 B)][K1Args x max_reqs][K1Work x max_work]
  char* h_table = nullptr;  // pinned copy written before each replay
  float4* chaninfo = nullptr;
  float4* rowinfo = nullptr;
  std::vector<uint64_t> reqs;
  bool busy = false;
};

}  // namespace wn

struct wn_server {
  wn_ctx* ctx = nullptr;
  int max_inflight = 8;
  int max_reqs = 64;
  int max_work = 1 << 14;
  size_t table_bytes = 0;
  int max_rows = 0, max_chan = 0;
  char* pool = nullptr;
  size_t pool_bytes = 0;
  std::map<size_t, size_t> free_list;  // offset -> size
  std::vector<wn::ServeSlot> slots;
  std::map<uint64_t, wn::ServeReq> reqs;
  std::deque<uint64_t> queue;  // pending, in arrival order
  uint64_t next_ticket = 1;
  int admitted = 0;            // admitted and not yet released
  int batches = 0, max_running_batches = 0, max_batch_reqs = 0, launched = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;
};

namespace wn {

static double now_s(wn_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

static bool pool_alloc(wn_server* s, size_t bytes, size_t* off) {
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t base = it->first;
      s->free_list.erase(it);
      if (rest) s->free_list[base + bytes] = rest;
      return true;
    }
  }
  return false;
}

static void pool_free(wn_server* s, size_t off, size_t bytes) {
  auto it = s->free_list.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_list.erase(nx);
  }
  if (it != s->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_list.erase(it);
    }
  }
}

static size_t round_bytes(size_t b) { return (b + 255) & ~(size_t)255; }

// Build one batch from admitted requests and launch it on slot `k`. Called with the lock held.
static void launch_batch(wn_server* s, int k) {
  ServeSlot& sl = s->slots[k];
  int* n_work = reinterpret_cast<int*>(sl.h_table);
  K1Args* args = reinterpret_cast<K1Args*>(sl.h_table + 16);
  K1Work* work = reinterpret_cast<K1Work*>(sl.h_table + 16 + sizeof(K1Args) * s->max_reqs);
  int nreq = 0, nwork = 0;
  sl.reqs.clear();
  std::vector<uint64_t> shapes;
  for (auto& kv : s->reqs) {
    ServeReq& r = kv.second;
    if (r.state != RQ_ADMITTED) continue;
    if (nreq == s->max_reqs) break;
    float2* out = reinterpret_cast<float2*>(s->pool + r.off);
    const bool pg = r.M->n_point + r.M->n_gauss > 0 || r.M->n_shape == 0;
    if (pg) {
      int gx = 0, gy = 0;
      if (k1_batched_args(s->ctx, r.od, r.M, out, r.mode, r.pa, &args[nreq], &gx, &gy) != WN_OK) {
        r.state = RQ_FAILED;
        r.error = WN_EINVAL;
        continue;
      }
      if (nwork + gx * gy > s->max_work) {
        if (nwork == 0) {  // larger than any batch: refuse rather than stall the queue
          r.state = RQ_FAILED;
          r.error = WN_EBUSY;
        }
        continue;
      }
      for (int y = 0; y < gy; ++y)
        for (int x = 0; x < gx; ++x) work[nwork++] = K1Work{nreq, x, y};
      ++nreq;
    }
    r.state = RQ_RUNNING;
    r.batch = s->batches;
    r.t_launch = now_s(s);
    sl.reqs.push_back(r.ticket);
    if (r.M->n_shape > 0) shapes.push_back(r.ticket);
  }
  if (sl.reqs.empty()) return;
  *n_work = nwork;
  cudaError_t e = cudaGraphLaunch(sl.gexec, sl.st);  // copies the table, then the batched kernel
  for (uint64_t t : shapes) {
    ServeReq& r = s->reqs[t];
    const bool pg = r.M->n_point + r.M->n_gauss > 0;
    const int smode = pg ? (r.mode == OUT_PEEL ? OUT_SUBG : OUT_ACCUM) : r.mode;
    if (launch_shapelets_ws(s->ctx, r.od, r.M, reinterpret_cast<float2*>(s->pool + r.off), smode, r.pa, sl.chaninfo,
                            sl.rowinfo, sl.st) != WN_OK) {
      r.state = RQ_FAILED;
      r.error = WN_ECUDA;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.st);
  if (e != cudaSuccess) {
    for (uint64_t t : sl.reqs) {
      s->reqs[t].state = RQ_FAILED;
      s->reqs[t].error = WN_ECUDA;
    }
  }
  sl.busy = true;
  s->batches++;
  s->launched += (int)sl.reqs.size();
  s->max_batch_reqs = std::max(s->max_batch_reqs, (int)sl.reqs.size());
  int running = 0;
  for (auto& x : s->slots) running += x.busy ? 1 : 0;
  s->max_running_batches = std::max(s->max_running_batches, running);
}

static void scheduler(wn_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    // completions
    for (auto& sl : s->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      const double t = now_s(s);
      for (uint64_t tk : sl.reqs) {
        ServeReq& r = s->reqs[tk];
        if (r.state == RQ_RUNNING) {
          r.state = q == cudaSuccess ? RQ_DONE : RQ_FAILED;
          if (q != cudaSuccess) r.error = WN_ECUDA;
        }
        r.t_done = t;
      }
      sl.reqs.clear();
      sl.busy = false;
      progress = true;
    }
    // admission by slots and memory, in arrival order (a request that does not fit yet does not
    // block smaller ones behind it)
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      ServeReq& r = s->reqs[*it];
      if (r.state != RQ_PENDING) {
        it = s->queue.erase(it);
        continue;
      }
      size_t off = 0;
      if (s->admitted < s->max_inflight && pool_alloc(s, r.bytes, &off)) {
        r.off = off;
        r.has_mem = true;
        r.state = RQ_ADMITTED;
        r.t_admit = now_s(s);
        s->admitted++;
        it = s->queue.erase(it);
        progress = true;
      } else {
        ++it;
      }
    }
    // launch admitted work on a free stream
    bool have = false;
    for (auto& kv : s->reqs)
      if (kv.second.state == RQ_ADMITTED) {
        have = true;
        break;
      }
    if (have) {
      for (int k = 0; k < (int)s->slots.size(); ++k)
        if (!s->slots[k].busy) {
          launch_batch(s, k);
          progress = true;
          break;
        }
    }
    if (progress) s->cv.notify_all();
    s->cv.wait_for(lk, std::chrono::microseconds(progress ? 0 : 20));
  }
}

}  // namespace wn

using namespace wn;

extern "C" {

int wn_server_create(wn_ctx* ctx, int n_streams, size_t pool_bytes, int max_inflight, int max_rows, int max_chan,
                     wn_server** out) {
  if (!ctx || !out) return set_error(WN_EINVAL, "NULL argument");
  *out = nullptr;
  if (n_streams < 1 || n_streams > 16 || max_inflight < 1 || max_rows < 1 || max_chan < 1 || pool_bytes < 256)
    return set_error(WN_EINVAL, "server sizes out of range");
  cudaSetDevice(ctx->device);
  wn_server* s = new wn_server();
  s->ctx = ctx;
  s->max_inflight = max_inflight;
  s->max_reqs = std::max(1, std::min(max_inflight, 256));
  s->max_rows = max_rows;
  s->max_chan = max_chan;
  s->table_bytes = 16 + sizeof(K1Args) * s->max_reqs + sizeof(K1Work) * s->max_work;
  s->pool_bytes = pool_bytes & ~(size_t)255;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaMalloc(&s->pool, s->pool_bytes);
  if (e != cudaSuccess) {
    delete s;
    return set_error(WN_ENOMEM, std::string("server pool: ") + cudaGetErrorString(e));
  }
  s->free_list[0] = s->pool_bytes;
  const size_t chan_bytes = round_bytes((size_t)max_chan * sizeof(float4));
  const int grid = ctx->num_sms * 2;
  s->slots.resize(n_streams);
  for (auto& sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_table, s->table_bytes);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_table, s->table_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&sl.chaninfo, chan_bytes + (size_t)max_rows * sizeof(float4));
    if (e == cudaSuccess) sl.rowinfo = reinterpret_cast<float4*>(reinterpret_cast<char*>(sl.chaninfo) + chan_bytes);
    if (e == cudaSuccess) {
      // graph per stream: copy of the work table from pinned memory, then the batched kernel
      cudaGraph_t g = nullptr;
      e = k1_batched_setup();
      if (e == cudaSuccess) e = cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaMemcpyAsync(sl.d_table, sl.h_table, s->table_bytes, cudaMemcpyHostToDevice, sl.st);
        const K1Args* d_args = reinterpret_cast<const K1Args*>(sl.d_table + 16);
        const K1Work* d_work = reinterpret_cast<const K1Work*>(sl.d_table + 16 + sizeof(K1Args) * s->max_reqs);
        k1_batched_launch(d_args, d_work, reinterpret_cast<const int*>(sl.d_table), grid, sl.st);
        e = cudaStreamEndCapture(sl.st, &g);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.gexec, g, 0);
      if (g) cudaGraphDestroy(g);
    }
  }
  if (e != cudaSuccess) {
    for (auto& sl : s->slots) {
      if (sl.gexec) cudaGraphExecDestroy(sl.gexec);
      if (sl.st) cudaStreamDestroy(sl.st);
      if (sl.done) cudaEventDestroy(sl.done);
      cudaFree(sl.d_table);
      if (sl.h_table) cudaFreeHost(sl.h_table);
      cudaFree(sl.chaninfo);
    }
    cudaFree(s->pool);
    delete s;
    return set_error(WN_ECUDA, std::string("server setup: ") + cudaGetErrorString(e));
  }
  s->worker = std::thread(scheduler, s);
  *out = s;
  return WN_OK;
}

void wn_server_destroy(wn_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  for (auto& sl : s->slots) {
    cudaStreamSynchronize(sl.st);
    cudaGraphExecDestroy(sl.gexec);
    cudaStreamDestroy(sl.st);
    cudaEventDestroy(sl.done);
    cudaFree(sl.d_table);
    cudaFreeHost(sl.h_table);
    cudaFree(sl.chaninfo);
  }
  cudaFree(s->pool);
  delete s;
}

int wn_server_submit(wn_server* s, const wn_obs* obs, int model_id, int peel, const void* gains_c64, int gains_t,
                     int gains_f, const void* data_c64, uint64_t* ticket) {
  if (!s || !ticket) return set_error(WN_EINVAL, "NULL argument");
  *ticket = 0;
  ServeReq r;
  if (!obs) return set_error(WN_EINVAL, "obs is NULL");
  // validation shared with the single-request entry points
  if (obs->n_ant < 2 || obs->n_base < 1 || obs->n_time < 1 || obs->n_chan < 1 || !obs->uvw || !obs->freq_hz ||
      !obs->ant1 || !obs->ant2 || !(obs->freq0_hz > 0.0))
    return set_error(WN_EINVAL, "invalid observation");
  if (!(obs->chan_spacing_hz > 0.0) && obs->n_chan > 1)
    return set_error(WN_EINVAL, "served observations need uniformly spaced channels");
  r.od.n_ant = obs->n_ant;
  r.od.n_base = obs->n_base;
  r.od.n_time = obs->n_time;
  r.od.n_chan = obs->n_chan;
  r.od.n_rows = obs->n_base * obs->n_time;
  r.od.uvw = obs->uvw;
  r.od.freq = obs->freq_hz;
  r.od.ant1 = obs->ant1;
  r.od.ant2 = obs->ant2;
  r.od.dec0 = obs->dec0;
  r.od.nu0 = obs->freq0_hz;
  r.od.dnu = obs->chan_spacing_hz;
  r.od.uniform = true;
  if (r.od.n_rows > s->max_rows || r.od.n_chan > s->max_chan)
    return set_error(WN_EINVAL, "observation larger than the server's row / channel tables");
  if (peel) {
    if (!gains_c64 || !data_c64 || !(gains_t == 1 || gains_t == obs->n_time) || !(gains_f == 1 || gains_f == obs->n_chan))
      return set_error(WN_EINVAL, "peel request needs data and gains [1|T][1|F][A]");
    r.pa.data = static_cast<const float2*>(data_c64);
    r.pa.gains = static_cast<const float2*>(gains_c64);
    r.pa.ant1 = obs->ant1;
    r.pa.ant2 = obs->ant2;
    r.pa.gt = gains_t;
    r.pa.gf = gains_f;
    r.pa.n_ant = obs->n_ant;
  }
  r.mode = peel ? OUT_PEEL : OUT_STORE;
  r.bytes = round_bytes((size_t)r.od.n_rows * r.od.n_chan * sizeof(float2));
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->ctx->models.find(model_id);
  if (it == s->ctx->models.end()) return set_error(WN_ENOTFOUND, "unknown model id");
  r.M = it->second;
  if (r.bytes > s->pool_bytes) return set_error(WN_EBUSY, "request larger than the server's memory pool");
  r.ticket = s->next_ticket++;
  r.t_submit = now_s(s);
  s->reqs[r.ticket] = r;
  s->queue.push_back(r.ticket);
  *ticket = r.ticket;
  s->cv.notify_all();
  return WN_OK;
}

// info: [t_submit, t_admit, t_launch, t_done] seconds on the server clock, then batch index.
int wn_server_poll(wn_server* s, uint64_t ticket, int* state, void** vis_out, double* info) {
  if (!s || !state) return set_error(WN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
  const ServeReq& r = it->second;
  *state = r.state;
  if (vis_out) *vis_out = r.state == RQ_DONE ? static_cast<void*>(s->pool + r.off) : nullptr;
  if (info) {
    info[0] = r.t_submit;
    info[1] = r.t_admit;
    info[2] = r.t_launch;
    info[3] = r.t_done;
    info[4] = r.batch;
  }
  return r.state == RQ_FAILED ? set_error(r.error, "request failed") : WN_OK;
}

int wn_server_wait(wn_server* s, uint64_t ticket, double timeout_s, void** vis_out, double* info) {
  if (!s) return set_error(WN_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
    const int st = it->second.state;
    if (st == RQ_DONE || st == RQ_FAILED || st == RQ_CANCELLED) break;
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) return set_error(WN_ETIMEOUT, "wait timed out");
  }
  lk.unlock();
  int state = 0;
  return wn_server_poll(s, ticket, &state, vis_out, info);
}

int wn_server_release(wn_server* s, uint64_t ticket) {
  if (!s) return set_error(WN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
  ServeReq& r = it->second;
  if (r.state == RQ_RUNNING || r.state == RQ_ADMITTED) return set_error(WN_EBUSY, "request still on the GPU");
  if (r.has_mem) {
    pool_free(s, r.off, r.bytes);
    s->admitted--;
  }
  s->reqs.erase(it);
  s->cv.notify_all();
  return WN_OK;
}

int wn_server_copy(wn_server* s, uint64_t ticket, void* dst, void* stream) {
  if (!s || !dst) return set_error(WN_EINVAL, "NULL argument");
  const void* src = nullptr;
  size_t bytes = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
    if (it->second.state != RQ_DONE) return set_error(WN_EBUSY, "request not done");
    src = s->pool + it->second.off;
    bytes = (size_t)it->second.od.n_rows * it->second.od.n_chan * sizeof(float2);
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("copy result: ") + cudaGetErrorString(e));
  return WN_OK;
}

int wn_server_cancel(wn_server* s, uint64_t ticket) {
  if (!s) return set_error(WN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
  if (it->second.state != RQ_PENDING) return set_error(WN_EBUSY, "request already admitted");
  it->second.state = RQ_CANCELLED;
  return WN_OK;
}

// stats: [batches, max batches on the GPU at once, most requests in one batch, requests launched,
//         requests admitted now, free pool bytes]
int wn_server_stats(wn_server* s, double* stats) {
  if (!s || !stats) return set_error(WN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  size_t free_b = 0;
  for (auto& kv : s->free_list) free_b += kv.second;
  stats[0] = s->batches;
  stats[1] = s->max_running_batches;
  stats[2] = s->max_batch_reqs;
  stats[3] = s->launched;
  stats[4] = s->admitted;
  stats[5] = (double)free_b;
  return WN_OK;
}

}  // extern "C"
