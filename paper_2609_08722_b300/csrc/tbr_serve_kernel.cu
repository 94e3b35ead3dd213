// Persistent serving kernel (continuous batching of hard renders, edits and
// soft render + adjoint requests).  The host copies request descriptors into a
// ring in device memory and then advances a published-item counter in mapped
// pinned memory (read only when a CTA runs out of known work); each CTA claims
// the next item with a compare-and-swap on a device counter and runs it: a
// 32x8 hard tile, or a group of 32x16 soft tiles (two pixels per thread)
// fused with the MSE seed and the replay adjoint.  The CTA that finishes a
// request's last item signals completion through mapped memory (the host then
// runs the fixed-order gradient sums of a soft request as ordinary kernels).
// Every wait is bounded; the kernel exits after idle_ns without work and the
// host relaunches it when new work is published.
#include "tbr_serve.h"
#include "tbr_pair.cuh"

namespace tbr {

namespace {

constexpr int kServeCH = 32;

__device__ __forceinline__ long long ld_volatile_ll(const volatile long long* p) { return *p; }

// Two CTAs per SM at 128 registers (at three CTAs per SM the paired adjoint's
// spills cost the soft requests more than the third CTA gains the hard ones).
// The soft items run the blocked stroke loops of the standalone kernels (the
// adjoint also two strokes per iteration); their second loop copies cost a few
// spilled registers and still win.  The host leaves four CTA slots of the
// machine to the packing, edit and epilogue kernels of other requests.
__global__ void __launch_bounds__(kTileThreads, 2) k_serve(ServeArgs a) {
  __shared__ __align__(128) float sbuf[2 * kServeCH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  __shared__ float red[2][kTileThreads / 32][kServeCH * 8];
  __shared__ __align__(16) f2 pbuf[kServeCH * kPairRec];
  __shared__ __align__(16) f2 pext[kServeCH * kPairExt];
  __shared__ double lsum[kTileThreads / 32];
  __shared__ ServeDesc sd;
  __shared__ long long s_item;
  __shared__ long long s_cursor;
  __shared__ int s_last;
  __shared__ long long s_pub;        // last published count seen (host memory is read only when exhausted)
  __shared__ long long s_have;       // seq of the descriptor cached in sd (-1: none)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ChunkRing<kServeCH> ring;
  ring.init(sbuf, sbar);
  if (threadIdx.x == 0) {
    s_cursor = a.first_seq;
    s_pub = 0;
    s_have = -1;
  }
  const size_t cta = blockIdx.x;
  while (true) {
    // ---- claim the next published item (thread 0).  The kernel closes only when
    // every CTA has been idle (no claimable item) for idle_ns, so no CTA leaves
    // while others still run and new work would find the GPU partly empty.
    if (threadIdx.x == 0) {
      long long got = -1;
      uint64_t idle0 = 0;
      bool counted_idle = false;
      unsigned backoff = 256;
      for (uint32_t it = 0;; ++it) {
        if (*reinterpret_cast<volatile int*>(a.closing)) break;
        const long long cur = static_cast<long long>(
            atomicAdd(reinterpret_cast<unsigned long long*>(a.next_item), 0ull));
        if (cur < s_pub) {
          if (static_cast<long long>(atomicCAS(reinterpret_cast<unsigned long long*>(a.next_item),
                                               static_cast<unsigned long long>(cur),
                                               static_cast<unsigned long long>(cur + 1))) == cur) {
            got = cur;
            break;
          }
          continue;
        }
        // nothing known to be claimable: look at the host's counter (mapped memory), back off
        const long long pub = ld_volatile_ll(&a.ctl->published);
        if (pub > s_pub) {
          s_pub = pub;
          backoff = 256;
          continue;
        }
        if (a.ctl->stop) {
          atomicExch(a.closing, 1);
          break;
        }
        if (!counted_idle) {
          atomicAdd(a.idle_ctas, 1);
          counted_idle = true;
          idle0 = global_timer_ns();
        } else if (global_timer_ns() - idle0 > a.idle_ns &&
                   atomicAdd(a.idle_ctas, 0) == static_cast<int>(gridDim.x)) {
          atomicExch(a.closing, 1);
          break;
        }
        __nanosleep(backoff);
        backoff = min(backoff * 2u, 32768u);
      }
      if (got >= 0 && counted_idle) atomicSub(a.idle_ctas, 1);
      s_item = got;
      if (got >= 0 && !(s_have >= 0 && got >= sd.item_base && got < sd.item_base + sd.n_items)) {
        // locate the request (device-memory ring, L1 bypassed): items are published
        // contiguously in request order; an entry whose seq differs from the cursor was
        // recycled (its request is complete), and an entry being rewritten belongs to a
        // request whose items are not published yet, so it cannot contain `got`
        long long c = s_cursor;
        for (int guard = 0; guard < 4 * kServeRing; ++guard) {
          const ServeDesc* e = &a.ring[c % kServeRing];
          const long long sq = __ldcg(&e->seq);
          const long long base = __ldcg(&e->item_base);
          const int cnt = __ldcg(&e->n_items);
          if (sq == c && got >= base && got < base + cnt) break;
          ++c;
        }
        s_cursor = c;
        const unsigned int* src = reinterpret_cast<const unsigned int*>(&a.ring[c % kServeRing]);
        unsigned int* dst = reinterpret_cast<unsigned int*>(&sd);
        for (size_t w = 0; w < sizeof(ServeDesc) / 4; ++w) dst[w] = __ldcg(src + w);
        s_have = c;
      }
    }
    __syncthreads();
    const long long item = s_item;
    if (item < 0) break;
    const ServeDesc& d = sd;
    const long long local = item - d.item_base;
    bool ok = true;
    // the request's ready word (if any): thread 0 waits for it, at most
    // ready_wait_ns; a request that already timed out skips the wait and the work
    if (threadIdx.x == 0) {
      int go = 1;
      if (d.ready) {
        go = d.status[ST_TIMEOUT] == 0ull ? 1 : 0;
        if (go && *d.ready == 0) {
          const uint64_t t0 = global_timer_ns();
          unsigned backoff = 64;
          while (*d.ready == 0) {
            if (global_timer_ns() - t0 > d.ready_wait_ns) {
              atomicAdd(d.status + ST_TIMEOUT, 1ull);
              go = 0;
              break;
            }
            __nanosleep(backoff);
            backoff = min(backoff * 2u, 4096u);
          }
        }
        __threadfence();  // inputs written before the ready word are seen after it
      }
      s_last = go;
    }
    __syncthreads();
    const bool run_item = s_last != 0;
    __syncthreads();  // s_last is reused at completion
    if (!run_item) {
      // nothing of the item is computed; its status reports the timeout (a soft
      // request's loss part is poisoned, so its loss and gradients come out NaN)
      if (d.kind != kServeHard && threadIdx.x == 0) d.loss_part[local] = __longlong_as_double(0x7ff8000000000000ll);
    } else if (d.kind == kServeHard) {
      const bool poison = d.status[ST_INVALID] != 0ull;
      unsigned band = 0, visited = 0;
      bool background = false;
      ok = hard_tile<kServeCH>(ring, d.packed, d.n, static_cast<int>(local), d.W, d.H, d.bg, poison, d.out_rgb,
                               d.out_idx, band, visited, background, d.status);
    } else {
      // soft render + MSE seed + replay adjoint over 32x16 tiles local, local + G, ...
      const int ntiles = pair_tile_count(d.W, d.H);
      constexpr size_t kSlot = 2 * kTileThreads;  // pixels per record slot of one CTA
      const RecordView rv{a.rec + cta * a.cap * kSlot, a.rec_i + cta * a.cap * kSlot,
                          a.ckpt + cta * a.nck_max * kSlot, a.ck_lt + cta * a.nck_max * kSlot, kSlot, 0, d.cap,
                          d.ck};
      const size_t off[2] = {static_cast<size_t>(threadIdx.x), static_cast<size_t>(threadIdx.x) + kTileThreads};
      float* slice = d.partial + static_cast<size_t>(local) * d.n * 8;
      const bool skip = d.status[ST_INVALID] != 0ull;
      double lacc = 0.0;
      unsigned drift = 0, ovf = 0;
      bool first = true;
      for (int tile = static_cast<int>(local); tile < ntiles; tile += d.n_items) {
        int px, py0;
        pair_tile_pixel(tile, d.W, px, py0);
        bool valid[2];
        size_t p[2];
        float x0[2], y0[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int py = py0 + c;
          valid[c] = px < d.W && py < d.H && !skip;
          p[c] = valid[c] ? static_cast<size_t>(py) * d.W + px : 0;
          x0[c] = (static_cast<float>(px) + 0.5f) / static_cast<float>(d.W);
          y0[c] = (static_cast<float>(py) + 0.5f) / static_cast<float>(d.H);
        }
        PixelState st[2];
        if (!soft_forward_tile2<kServeCH, true>(ring, d.packed, d.n, valid, x0, y0, rv, off, pbuf, pext, st, d.status)) {
          ok = false;
          break;
        }
        float lC[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (!valid[c]) continue;
          const size_t q = p[c];
          const float T0 = ex2_a(st[c].lt);
          const float R0 = fmaf(T0, d.bg[0], st[c].C0), R1 = fmaf(T0, d.bg[1], st[c].C1),
                      R2 = fmaf(T0, d.bg[2], st[c].C2);
          if (d.out_rgb) {
            d.out_rgb[3 * q + 0] = R0;
            d.out_rgb[3 * q + 1] = R1;
            d.out_rgb[3 * q + 2] = R2;
          }
          const float e0 = R0 - d.target[3 * q + 0], e1 = R1 - d.target[3 * q + 1], e2 = R2 - d.target[3 * q + 2];
          lacc += static_cast<double>(e0) * e0 + static_cast<double>(e1) * e1 + static_cast<double>(e2) * e2;
          lC[c][0] = d.seed_scale * e0; lC[c][1] = d.seed_scale * e1; lC[c][2] = d.seed_scale * e2;
          if (st[c].cnt > d.cap) ++ovf;
        }
        if (!backward_tile2<kServeCH, false, 2, false, true>(ring, d.packed, d.n, valid, st, lC, d.bg, rv, off, pbuf,
                                                             red, slice, first, drift, d.status)) {
          ok = false;
          break;
        }
        first = false;
      }
      if (first && ok) {  // a group with no tile (cannot happen: n_items <= ntiles) keeps a zero slice
        for (int t = threadIdx.x; t < d.n * 8; t += blockDim.x) slice[t] = 0.0f;
      }
      for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
      if (lane == 0) lsum[warp] = lacc;
      const unsigned osum = __reduce_add_sync(0xffffffffu, ovf);
      if (lane == 0 && osum) atomicAdd(d.status + ST_OVERFLOW, static_cast<unsigned long long>(osum));
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kTileThreads / 32; ++w) s += lsum[w];
        d.loss_part[local] = s;
      }
    }
    (void)ok;  // a failing bounded wait has already set the request's timeout word
    // ---- completion
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const int done = atomicAdd(a.items_done + d.slot, 1) + 1;
      s_last = (done == d.n_items) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
      // all items of the request are done: signal the host (which runs the
      // gradient epilogue of soft requests with ordinary kernels)
      if (threadIdx.x == 0) {
        a.items_done[d.slot] = 0;  // the slot is reused by a later request
        __threadfence_system();
        a.ctl->done[d.slot] = d.seq;
        __threadfence_system();
      }
    }
    __syncthreads();
  }
}

}  // namespace

int serve_grid() {
  static PerDeviceInt cache;
  const int per_sm = cache.get([](int) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_serve, kTileThreads, 0) != cudaSuccess || b < 1) b = 1;
    return b;
  });
  // leave a few CTA slots free so packing, edit and epilogue kernels of other requests can run
  // alongside (with none free they queue behind the persistent CTAs: 93 instead of 99 req/s)
  const int g = per_sm * device_sm_count();
  return g > 16 ? g - 4 : g;
}

cudaError_t launch_serve(const ServeArgs& a, cudaStream_t st) {
  KernelTimer kt(TBR_K_SERVE, st);
  k_serve<<<a.grid, kTileThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tbr
