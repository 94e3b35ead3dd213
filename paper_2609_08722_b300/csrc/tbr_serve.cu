// Serving (continuous batching) host side: resident programs, a request queue
// with admission by device memory, edit preparation (recolour, reorder, stroke
// insert; Sec. 7 "program edits"), publication of work to the persistent
// kernel (tbr_serve_kernel.cu) and completion tracking with latencies.
//
// A worker thread admits queued requests in arrival order while slots, ring
// entries and the memory cap allow; admission packs the (possibly edited)
// program on a side stream and publishes the request's work items.  Requests
// that arrive while others are on the GPU are admitted as soon as resources
// free up and their items interleave with the running ones in the same
// persistent launch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "tbr_host.h"
#include "tbr_serve.h"
#include "tbr_tile.cuh"

namespace tbr {
namespace {

using Clock = std::chrono::steady_clock;

__global__ void k_edit(const float* __restrict__ src, int n, int k, int kind, int a, int b, int start,
                       const float* __restrict__ ins, int ins_pal, float* __restrict__ dst, int n_out) {
  // src / dst: [cx | cy | theta | length | half_width | logits (n k)]
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out) return;
  int from = i;           // source stroke of output stroke i (-1 = the inserted stroke)
  if (kind == TBR_REQ_REORDER) {
    if (i >= start && i < start + b) from = start + (start + b - 1 - i);
  } else if (kind == TBR_REQ_INSERT) {
    if (i == start) from = -1;
    else if (i > start) from = i - 1;
  }
  for (int f = 0; f < 5; ++f)
    dst[static_cast<size_t>(f) * n_out + i] = from >= 0 ? src[static_cast<size_t>(f) * n + from] : ins[f];
  for (int q = 0; q < k; ++q) {
    float z;
    if (from < 0) {
      z = (q == ins_pal) ? 6.0f : 0.0f;  // one-hot assignment of the inserted stroke
    } else {
      int qq = q;
      if (kind == TBR_REQ_RECOLOUR && i >= start) qq = (q == a) ? b : (q == b) ? a : q;  // swap entries a, b
      z = src[5 * static_cast<size_t>(n) + static_cast<size_t>(from) * k + qq];
    }
    dst[5 * static_cast<size_t>(n_out) + static_cast<size_t>(i) * k + q] = z;
  }
}

struct Program {
  int n = 0, k = 0;
  float* params = nullptr;   // [5n + nk]
  float* palette = nullptr;  // [k][3]
  float bg[3] = {1, 1, 1};
  float color_temp = 1.0f;
  size_t bytes = 0;
};

struct Request {
  uint64_t id = 0;
  tbr_request req{};
  int kind = kServeHard;
  int n = 0, k = 0;
  long long seq = -1;
  int slot = -1;
  int n_items = 0;
  size_t bytes = 0;
  int state = 0;  // 0 queued, 4 staged (preparation enqueued), 1 running, 3 finishing, 2 done
  cudaEvent_t ready = nullptr;     // inputs ready on the caller's stream
  cudaEvent_t staged = nullptr;    // preparation (edit, pack, descriptor copy) done
  cudaEvent_t finished = nullptr;  // epilogue and status copy done
  tbr_status result = TBR_OK;
  Clock::time_point t_submit, t_admit, t_done;
  // resources
  float* derived = nullptr;  // edited program [5n + nk]
  float* packed = nullptr;
  float* probs = nullptr;
  unsigned long long* status = nullptr;
  float* partial = nullptr;
  double* loss_part = nullptr;
  float* grad8 = nullptr;
};

}  // namespace
}  // namespace tbr

struct tbr_server {
  tbr_serve_config cfg;
  int device = 0;
  cudaStream_t kstream = nullptr;  // persistent kernel
  cudaStream_t astream = nullptr;  // admission (packing, edits, memsets)
  tbr::ServeCtl* ctl = nullptr;    // mapped pinned (host view)
  tbr::ServeCtl* ctl_dev = nullptr;
  tbr::ServeDesc* ring_dev = nullptr;  // device memory
  tbr::ServeDesc* stage = nullptr;     // pinned host staging [kServeRing]
  unsigned long long* status_host = nullptr;  // pinned [kServeMaxSlots][ST_COUNT]
  long long* next_item = nullptr;
  int* items_done = nullptr;
  int* idle_flags = nullptr;       // [0] idle CTAs, [1] closing
  float4* rec = nullptr;
  int* rec_i = nullptr;
  float4* ckpt = nullptr;
  float* ck_lt = nullptr;
  size_t nck_max = 0;
  int grid = 0;
  size_t fixed_bytes = 0;
  // host state
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stopping = false;
  bool kernel_running = false;
  std::map<uint64_t, tbr::Program> programs;
  std::map<uint64_t, tbr::Request> requests;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> inflight;    // staged, running or finishing, in admission order
  std::vector<int> free_slots;
  uint64_t next_prog_id = 1, next_req_id = 1;
  long long next_seq = 0;
  long long published = 0;     // items visible to the kernel
  long long staged_items = 0;  // items of admitted requests (published or about to be)
  long long oldest_unfinished_seq = 0;
  size_t bytes_in_use = 0;
  int64_t kernel_launches = 0, completed = 0, admitted = 0, refused = 0;
  tbr_status fatal = TBR_OK;
};

namespace tbr {
namespace {

size_t request_bytes(const tbr_server* s, const tbr_request& r, int n, int k) {
  const size_t n_out = (r.kind == TBR_REQ_INSERT) ? static_cast<size_t>(n) + 1 : static_cast<size_t>(n);
  size_t b = n_out * kRec * 4 + ST_COUNT * 8;
  if (r.kind >= TBR_REQ_RECOLOUR) b += (5 * n_out + n_out * k) * 4;
  if (r.kind == TBR_REQ_SOFT_ADJOINT) {
    const int groups = std::min(pair_tile_count(r.W, r.H), s->grid);
    b += n_out * k * 4 + static_cast<size_t>(groups) * n_out * 32 + static_cast<size_t>(groups) * 8 + n_out * 32;
  }
  return b;
}

void release_request(tbr_server* s, Request& q) {
  cudaStream_t st = s->astream;
  if (q.ready) { cudaEventDestroy(q.ready); q.ready = nullptr; }
  if (q.staged) { cudaEventDestroy(q.staged); q.staged = nullptr; }
  if (q.finished) { cudaEventDestroy(q.finished); q.finished = nullptr; }
  dfree(q.derived, st); dfree(q.packed, st); dfree(q.probs, st); dfree(q.status, st);
  dfree(q.partial, st); dfree(q.loss_part, st); dfree(q.grad8, st);
}

// Allocates, edits, packs and publishes one request.  Caller holds s->mu.
tbr_status admit(tbr_server* s, Request& q) {
  const Program& pg = s->programs.at(q.req.program);
  cudaStream_t st = s->astream;
  const tbr_request& r = q.req;
  const int n_out = (r.kind == TBR_REQ_INSERT) ? pg.n + 1 : pg.n;
  const int k = pg.k;
  q.n = n_out; q.k = k;
  q.kind = (r.kind == TBR_REQ_SOFT_ADJOINT) ? kServeSoft : kServeHard;
  // a hard request is one item per 32x8 tile; a soft request one item per CTA-sized
  // group of 32x16 tiles
  const int n_items = q.kind == kServeHard ? tile_count(r.W, r.H) : std::min(pair_tile_count(r.W, r.H), s->grid);
  // the caller's inputs (and the zeroing of its outputs, if any) precede the work
  cudaError_t e = q.ready ? cudaStreamWaitEvent(st, q.ready, 0) : cudaSuccess;
  const float* params = pg.params;
  if (e == cudaSuccess && r.kind >= TBR_REQ_RECOLOUR) {
    e = dalloc(&q.derived, 5 * static_cast<size_t>(n_out) + static_cast<size_t>(n_out) * k, st);
    float* ins = nullptr;
    if (e == cudaSuccess) e = dalloc(&ins, 8, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ins, r.insert_stroke, 5 * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_out > 0) {
      k_edit<<<(n_out + 127) / 128, 128, 0, st>>>(pg.params, pg.n, k, r.kind, r.edit_a, r.edit_b, r.edit_start, ins,
                                                   r.insert_palette, q.derived, n_out);
      e = cudaGetLastError();
    }
    dfree(ins, st);  // stream-ordered: after k_edit
    params = q.derived;
  }
  if (e == cudaSuccess) e = dalloc(&q.packed, static_cast<size_t>(n_out) * kRec, st);
  if (e == cudaSuccess) e = dalloc(&q.status, ST_COUNT, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(q.status, 0, ST_COUNT * sizeof(unsigned long long), st);
  if (q.kind == kServeSoft) {
    if (e == cudaSuccess) e = dalloc(&q.probs, static_cast<size_t>(n_out) * k, st);
    if (e == cudaSuccess) e = dalloc(&q.partial, static_cast<size_t>(n_items) * n_out * 8, st);
    if (e == cudaSuccess) e = dalloc(&q.loss_part, static_cast<size_t>(n_items), st);
    if (e == cudaSuccess) e = dalloc(&q.grad8, static_cast<size_t>(n_out) * 8, st);
  }
  tbr_program view{};
  view.n = n_out; view.k = k;
  const size_t nn = static_cast<size_t>(n_out);
  view.cx = params; view.cy = params + nn; view.theta = params + 2 * nn; view.length = params + 3 * nn;
  view.half_width = params + 4 * nn; view.logits = params + 5 * nn; view.palette = pg.palette;
  for (int c = 0; c < 3; ++c) view.background[c] = pg.bg[c];
  view.color_temp = pg.color_temp;
  const bool soft = q.kind == kServeSoft;
  PackArgs pa{&view, n_out, soft ? r.tau : 0.0f, soft ? r.tau_min : 1.0f, (!soft && r.snap) ? 1 : 0, q.packed,
              soft ? q.probs : nullptr, q.status};
  if (e == cudaSuccess) e = launch_pack(pa, st);
  if (e != cudaSuccess) {
    release_request(s, q);
    return cuda_fail(e, "serve: admitting a request");
  }
  // slot + ring entry
  q.slot = s->free_slots.back();
  s->free_slots.pop_back();
  q.seq = s->next_seq++;
  ServeDesc& d = s->stage[q.seq % kServeRing];
  std::memset(&d, 0, sizeof(d));
  d.seq = q.seq;
  d.item_base = s->staged_items;
  d.kind = q.kind; d.n = n_out; d.k = k; d.W = r.W; d.H = r.H;
  d.n_items = n_items; d.slot = q.slot; d.ck = s->cfg.checkpoint_every; d.cap = s->cfg.record_capacity;
  for (int c = 0; c < 3; ++c) d.bg[c] = pg.bg[c];
  d.inv_tc = 1.0f / pg.color_temp;
  d.seed_scale = 2.0f / (3.0f * static_cast<float>(r.W) * static_cast<float>(r.H));
  d.packed = q.packed; d.out_rgb = r.out_rgb; d.out_idx = soft ? nullptr : r.out_idx; d.target = r.target;
  d.partial = q.partial; d.loss_part = q.loss_part; d.probs = q.probs; d.palette = pg.palette;
  d.grad8 = q.grad8; d.out_grad = r.out_grad; d.out_loss = r.out_loss; d.status = q.status;
  d.ready = reinterpret_cast<const volatile int*>(r.ready);
  d.ready_wait_ns = static_cast<unsigned long long>(s->cfg.ready_wait_us) * 1000ull;
  e = cudaMemcpyAsync(s->ring_dev + (q.seq % kServeRing), &d, sizeof(ServeDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.staged, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(q.staged, st);
  if (e != cudaSuccess) {
    s->free_slots.push_back(q.slot);
    release_request(s, q);
    return cuda_fail(e, "serve: staging a request");
  }
  s->staged_items += n_items;  // published once the staged event completes (in order)
  q.n_items = n_items;
  q.state = 4;
  q.t_admit = Clock::now();
  s->bytes_in_use += q.bytes;
  ++s->admitted;
  return TBR_OK;
}

void ensure_kernel(tbr_server* s) {
  if (s->kernel_running) {
    if (cudaStreamQuery(s->kstream) == cudaSuccess) s->kernel_running = false;
  }
  bool running_work = false;
  for (uint64_t id : s->inflight)
    if (s->requests.at(id).state == 1) running_work = true;
  if (s->kernel_running || !running_work) return;
  ServeArgs a;
  a.ctl = s->ctl_dev; a.ring = s->ring_dev; a.next_item = s->next_item; a.items_done = s->items_done;
  a.idle_ctas = s->idle_flags; a.closing = s->idle_flags + 1;
  a.rec = s->rec; a.rec_i = s->rec_i; a.ckpt = s->ckpt; a.ck_lt = s->ck_lt;
  a.cap = s->cfg.record_capacity; a.nck_max = s->nck_max;
  a.first_seq = s->oldest_unfinished_seq;
  a.idle_ns = static_cast<unsigned long long>(s->cfg.idle_exit_us) * 1000ull;
  a.grid = s->grid;
  if (cudaMemsetAsync(s->idle_flags, 0, 2 * sizeof(int), s->kstream) != cudaSuccess ||
      launch_serve(a, s->kstream) != cudaSuccess) {
    s->fatal = TBR_ERR_CUDA;
    return;
  }
  s->kernel_running = true;
  ++s->kernel_launches;
}

void worker_main(tbr_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stopping) {
    bool progress = false;
    // publish staged requests in admission order once their preparation has run
    for (uint64_t id : s->inflight) {
      Request& q = s->requests.at(id);
      if (q.state == 1 || q.state == 3) continue;
      if (q.state != 4 || cudaEventQuery(q.staged) != cudaSuccess) break;
      s->published += q.n_items;
      std::atomic_thread_fence(std::memory_order_seq_cst);
      s->ctl->published = s->published;
      std::atomic_thread_fence(std::memory_order_seq_cst);
      q.state = 1;
      progress = true;
    }
    // completions
    for (size_t j = 0; j < s->inflight.size();) {
      Request& q = s->requests.at(s->inflight[j]);
      bool finished = false;
      if (q.state == 1 && s->ctl->done[q.slot] == q.seq) {
        cudaError_t e = cudaSuccess;
        if (q.kind == kServeSoft) {
          // fixed-order sum of the group slices, colour chain rule and loss, on ordinary kernels
          const Program& pg = s->programs.at(q.req.program);
          const size_t n = static_cast<size_t>(q.n);
          EpilogueArgs ea;
          ea.partial = q.partial; ea.grid = q.n_items; ea.n = q.n; ea.k = q.k;
          ea.packed = q.packed; ea.probs = q.probs; ea.palette = pg.palette;
          ea.inv_color_temp = 1.0f / pg.color_temp; ea.grad8 = q.grad8;
          float* g = q.req.out_grad;
          ea.g_cx = g; ea.g_cy = g + n; ea.g_th = g + 2 * n; ea.g_len = g + 3 * n; ea.g_r = g + 4 * n;
          ea.g_logits = g + 5 * n; ea.g_pal = nullptr; ea.status = q.status;
          e = launch_backward_epilogue(ea, s->astream);
          if (e == cudaSuccess && q.req.out_loss)
            e = launch_loss_final(q.loss_part, q.n_items, 3ll * q.req.W * q.req.H, q.req.out_loss, s->astream);
        }
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(s->status_host + static_cast<size_t>(q.slot) * ST_COUNT, q.status,
                              ST_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->astream);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.finished, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(q.finished, s->astream);
        if (e != cudaSuccess) {
          q.result = TBR_ERR_CUDA;
          finished = true;
        } else {
          q.state = 3;
        }
        progress = true;
      } else if (q.state == 3 && cudaEventQuery(q.finished) == cudaSuccess) {
        const unsigned long long* host = s->status_host + static_cast<size_t>(q.slot) * ST_COUNT;
        q.result = host[ST_INVALID] ? TBR_ERR_INVALID_ARG
                   : host[ST_OVERFLOW] ? TBR_ERR_OVERFLOW
                   : host[ST_TIMEOUT] ? TBR_ERR_TIMEOUT : TBR_OK;
        finished = true;
        progress = true;
      }
      if (finished) {
        q.t_done = Clock::now();
        q.state = 2;
        release_request(s, q);
        s->bytes_in_use -= q.bytes;
        s->free_slots.push_back(q.slot);
        ++s->completed;
        s->inflight.erase(s->inflight.begin() + j);
        s->cv.notify_all();
      } else {
        ++j;
      }
    }
    long long oldest = s->next_seq;
    for (uint64_t id : s->inflight) {
      const Request& q = s->requests.at(id);
      if (q.state == 1 || q.state == 4) oldest = std::min(oldest, q.seq);
    }
    s->oldest_unfinished_seq = oldest;
    // admissions, in arrival order
    while (!s->queue.empty() && !s->free_slots.empty() &&
           static_cast<int>(s->inflight.size()) < std::min(s->cfg.max_inflight, kServeRing - 1)) {
      Request& q = s->requests.at(s->queue.front());
      if (s->bytes_in_use + q.bytes > s->cfg.memory_cap_bytes && !s->inflight.empty()) break;  // wait for memory
      s->queue.pop_front();
      const tbr_status st = admit(s, q);
      if (st != TBR_OK) {
        q.result = st;
        q.state = 2;
        q.t_done = Clock::now();
        ++s->refused;
        s->cv.notify_all();
      } else {
        s->inflight.push_back(q.id);
        bool older = false;
        for (uint64_t id : s->inflight) {
          const int stt = s->requests.at(id).state;
          if (id != q.id && (stt == 1 || stt == 4)) older = true;
        }
        if (!older) s->oldest_unfinished_seq = q.seq;
      }
      progress = true;
    }
    ensure_kernel(s);
    if (!progress) {
      if (s->inflight.empty() && s->queue.empty()) {
        s->cv.wait_for(lk, std::chrono::milliseconds(5));
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
}

}  // namespace
}  // namespace tbr

using namespace tbr;

extern "C" {

void tbr_serve_default_config(tbr_serve_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->memory_cap_bytes = static_cast<size_t>(80) << 30;
  c->max_inflight = 64;
  c->max_strokes = 8192;
  c->checkpoint_every = 64;
  c->record_capacity = 64;
  c->idle_exit_us = 2000;
  c->ready_wait_us = 1000000;
}

tbr_status tbr_serve_create(const tbr_serve_config* cfg, tbr_server** out) {
  if (!out) return fail(TBR_ERR_INVALID_ARG, "server handle pointer is NULL");
  *out = nullptr;
  tbr_serve_config c;
  if (cfg) c = *cfg; else tbr_serve_default_config(&c);
  if (c.max_inflight < 1 || c.max_inflight > kServeMaxSlots || c.max_strokes < 1 || c.checkpoint_every < 1 ||
      c.record_capacity < 1 || c.idle_exit_us < 1 || c.ready_wait_us < 0)
    return fail(TBR_ERR_INVALID_ARG, "invalid serving configuration");
  tbr_server* s = new tbr_server();
  s->cfg = c;
  cudaGetDevice(&s->device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->astream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&s->ctl), sizeof(ServeCtl), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->ctl_dev), s->ctl, 0);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->ring_dev), sizeof(ServeDesc) * kServeRing);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&s->stage), sizeof(ServeDesc) * kServeRing, cudaHostAllocDefault);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&s->status_host),
                      sizeof(unsigned long long) * ST_COUNT * kServeMaxSlots, cudaHostAllocDefault);
  if (e == cudaSuccess) {
    std::memset(const_cast<ServeCtl*>(s->ctl), 0, sizeof(ServeCtl));
    for (int i = 0; i < kServeMaxSlots; ++i) s->ctl->done[i] = -1;
    std::vector<ServeDesc> init(kServeRing);
    std::memset(init.data(), 0, sizeof(ServeDesc) * kServeRing);
    for (int i = 0; i < kServeRing; ++i) init[i].seq = -1;
    e = cudaMemcpy(s->ring_dev, init.data(), sizeof(ServeDesc) * kServeRing, cudaMemcpyHostToDevice);
  }
  s->grid = serve_grid();
  s->nck_max = c.max_strokes > 1 ? static_cast<size_t>((c.max_strokes - 1) / c.checkpoint_every) : 0;
  const size_t per = static_cast<size_t>(s->grid) * 2 * kTileThreads;  // pixels per record slot, all CTAs
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->next_item), sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->items_done), sizeof(int) * kServeMaxSlots);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->idle_flags), 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->rec), sizeof(float4) * c.record_capacity * per);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->rec_i), sizeof(int) * c.record_capacity * per);
  if (e == cudaSuccess && s->nck_max)
    e = cudaMalloc(reinterpret_cast<void**>(&s->ckpt), sizeof(float4) * s->nck_max * per);
  if (e == cudaSuccess && s->nck_max)
    e = cudaMalloc(reinterpret_cast<void**>(&s->ck_lt), sizeof(float) * s->nck_max * per);
  if (e == cudaSuccess) e = cudaMemset(s->next_item, 0, sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(s->items_done, 0, sizeof(int) * kServeMaxSlots);
  if (e != cudaSuccess) {
    tbr_serve_destroy(s);
    return cuda_fail(e, "tbr_serve_create");
  }
  s->fixed_bytes = per * (20ull * c.record_capacity + 20ull * s->nck_max);
  for (int i = c.max_inflight - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return TBR_OK;
}

tbr_status tbr_serve_load_program(tbr_server* s, const tbr_program* prog, uint64_t* id) {
  if (!s || !id) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  tbr_status st = check_program(prog, prog ? prog->n : 0);
  if (st != TBR_OK) return st;
  if (prog->coupling) return fail(TBR_ERR_INVALID_ARG, "the server renders the capsule map (coupling must be NULL)");
  if (prog->n > s->cfg.max_strokes - 1)
    return fail(TBR_ERR_INVALID_ARG, "program of %d strokes exceeds the server's max_strokes - 1 = %d", prog->n,
                s->cfg.max_strokes - 1);
  Program pg;
  pg.n = prog->n; pg.k = prog->k;
  pg.color_temp = prog->color_temp;
  for (int c = 0; c < 3; ++c) pg.bg[c] = prog->background[c];
  const size_t n = pg.n, k = pg.k;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&pg.params), sizeof(float) * (5 * n + n * k + 1));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&pg.palette), sizeof(float) * 3 * k);
  const float* src[5] = {prog->cx, prog->cy, prog->theta, prog->length, prog->half_width};
  for (int f = 0; f < 5 && e == cudaSuccess && n > 0; ++f)
    e = cudaMemcpy(pg.params + f * n, src[f], n * 4, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(pg.params + 5 * n, prog->logits, n * k * 4, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pg.palette, prog->palette, k * 12, cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    if (pg.params) cudaFree(pg.params);
    if (pg.palette) cudaFree(pg.palette);
    return cuda_fail(e, "tbr_serve_load_program");
  }
  pg.bytes = 4 * (5 * n + n * k + 3 * k);
  std::lock_guard<std::mutex> lk(s->mu);
  *id = s->next_prog_id++;
  s->programs[*id] = pg;
  return TBR_OK;
}

tbr_status tbr_serve_submit(tbr_server* s, const tbr_request* r, uint64_t* req_id, void* stream) {
  if (!s || !r || !req_id) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != TBR_OK) return fail(s->fatal, "the server hit a CUDA error");
  auto it = s->programs.find(r->program);
  if (it == s->programs.end()) return fail(TBR_ERR_NOT_FOUND, "unknown program id %llu",
                                           static_cast<unsigned long long>(r->program));
  const Program& pg = it->second;
  if (r->kind < TBR_REQ_HARD || r->kind > TBR_REQ_INSERT) return fail(TBR_ERR_INVALID_ARG, "unknown request kind");
  tbr_status st = check_size(r->W, r->H);
  if (st != TBR_OK) return st;
  if (!r->out_rgb && r->kind != TBR_REQ_SOFT_ADJOINT) return fail(TBR_ERR_INVALID_ARG, "out_rgb is NULL");
  if (r->kind == TBR_REQ_SOFT_ADJOINT) {
    if (!r->target || !r->out_grad) return fail(TBR_ERR_INVALID_ARG, "soft requests need target and out_grad");
    if (!(r->tau >= 0.0f) || !(r->tau_min > 0.0f)) return fail(TBR_ERR_INVALID_ARG, "need tau >= 0, tau_min > 0");
    if (pg.n == 0) return fail(TBR_ERR_INVALID_ARG, "soft requests need a non-empty program");
  }
  if (r->kind == TBR_REQ_RECOLOUR &&
      (r->edit_a < 0 || r->edit_a >= pg.k || r->edit_b < 0 || r->edit_b >= pg.k || r->edit_start < 0))
    return fail(TBR_ERR_INVALID_ARG, "recolour needs palette entries in [0, k) and start >= 0");
  if (r->kind == TBR_REQ_REORDER && (r->edit_start < 0 || r->edit_b < 0 || r->edit_start + r->edit_b > pg.n))
    return fail(TBR_ERR_INVALID_ARG, "reorder window outside the program");
  if (r->kind == TBR_REQ_INSERT &&
      (r->edit_start < 0 || r->edit_start > pg.n || r->insert_palette < 0 || r->insert_palette >= pg.k ||
       !(r->insert_stroke[4] > 0.0f) || r->insert_stroke[3] < 0.0f))
    return fail(TBR_ERR_INVALID_ARG, "insert needs 0 <= index <= n, a palette entry and r > 0, L >= 0");
  const int n_out = r->kind == TBR_REQ_INSERT ? pg.n + 1 : pg.n;
  const size_t bytes = request_bytes(s, *r, pg.n, pg.k);
  if (bytes > s->cfg.memory_cap_bytes) {
    ++s->refused;
    return fail(TBR_ERR_ADMISSION, "request needs %zu bytes, above the memory cap %zu", bytes,
                static_cast<size_t>(s->cfg.memory_cap_bytes));
  }
  (void)n_out;
  Request q;
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    if (ev) cudaEventDestroy(ev);
    return cuda_fail(e, "tbr_serve_submit: recording the caller's stream");
  }
  q.ready = ev;
  q.id = s->next_req_id++;
  q.req = *r;
  q.bytes = bytes;
  q.t_submit = Clock::now();
  s->requests[q.id] = q;
  s->queue.push_back(q.id);
  *req_id = q.id;
  s->cv.notify_all();
  return TBR_OK;
}

tbr_status tbr_serve_poll(tbr_server* s, uint64_t req_id, int32_t* done, tbr_status* result) {
  if (!s || !done) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(req_id);
  if (it == s->requests.end()) return fail(TBR_ERR_NOT_FOUND, "unknown request id");
  *done = it->second.state == 2;
  if (result) *result = it->second.result;
  return TBR_OK;
}

tbr_status tbr_serve_wait(tbr_server* s, uint64_t req_id, int32_t timeout_ms, tbr_status* result) {
  if (!s) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(req_id);
  if (it == s->requests.end()) return fail(TBR_ERR_NOT_FOUND, "unknown request id");
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 3600000 : timeout_ms);
  while (s->requests.at(req_id).state != 2) {
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && s->requests.at(req_id).state != 2)
      return fail(TBR_ERR_TIMEOUT, "request %llu not finished within %d ms", static_cast<unsigned long long>(req_id),
                  timeout_ms);
  }
  if (result) *result = s->requests.at(req_id).result;
  return TBR_OK;
}

tbr_status tbr_serve_request_times(tbr_server* s, uint64_t req_id, double* queue_ms, double* latency_ms) {
  if (!s) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(req_id);
  if (it == s->requests.end()) return fail(TBR_ERR_NOT_FOUND, "unknown request id");
  const Request& q = it->second;
  if (q.state != 2) return fail(TBR_ERR_INVALID_ARG, "request not finished");
  using ms = std::chrono::duration<double, std::milli>;
  if (queue_ms) *queue_ms = q.seq >= 0 ? ms(q.t_admit - q.t_submit).count() : 0.0;
  if (latency_ms) *latency_ms = ms(q.t_done - q.t_submit).count();
  return TBR_OK;
}

tbr_status tbr_serve_release(tbr_server* s, uint64_t req_id) {
  if (!s) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(req_id);
  if (it == s->requests.end()) return fail(TBR_ERR_NOT_FOUND, "unknown request id");
  if (it->second.state != 2) return fail(TBR_ERR_INVALID_ARG, "request not finished");
  s->requests.erase(it);
  return TBR_OK;
}

tbr_status tbr_serve_stats(tbr_server* s, tbr_serve_counters* out) {
  if (!s || !out) return fail(TBR_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->refused = s->refused;
  out->queued = static_cast<int64_t>(s->queue.size());
  out->inflight = static_cast<int64_t>(s->inflight.size());
  out->kernel_launches = s->kernel_launches;
  out->bytes_in_use = static_cast<int64_t>(s->bytes_in_use);
  out->fixed_bytes = static_cast<int64_t>(s->fixed_bytes);
  out->persistent_ctas = s->grid;
  return TBR_OK;
}

void tbr_serve_destroy(tbr_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    if (s->ctl) s->ctl->stop = 1;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->kstream) cudaStreamSynchronize(s->kstream);
  if (s->astream) cudaStreamSynchronize(s->astream);
  for (auto& kv : s->requests)
    if (kv.second.state != 2) release_request(s, kv.second);
  if (s->astream) cudaStreamSynchronize(s->astream);
  for (auto& kv : s->programs) {
    cudaFree(kv.second.params);
    cudaFree(kv.second.palette);
  }
  if (s->next_item) cudaFree(s->next_item);
  if (s->items_done) cudaFree(s->items_done);
  if (s->idle_flags) cudaFree(s->idle_flags);
  if (s->rec) cudaFree(s->rec);
  if (s->rec_i) cudaFree(s->rec_i);
  if (s->ckpt) cudaFree(s->ckpt);
  if (s->ck_lt) cudaFree(s->ck_lt);
  if (s->ctl) cudaFreeHost(const_cast<ServeCtl*>(s->ctl));
  if (s->ring_dev) cudaFree(s->ring_dev);
  if (s->stage) cudaFreeHost(s->stage);
  if (s->status_host) cudaFreeHost(s->status_host);
  if (s->kstream) cudaStreamDestroy(s->kstream);
  if (s->astream) cudaStreamDestroy(s->astream);
  delete s;
}

}  // extern "C"
