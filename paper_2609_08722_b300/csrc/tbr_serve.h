// Internal structures shared by the serving kernel and its host side.
#pragma once

#include "tbr_internal.cuh"

namespace tbr {

constexpr int kServeRing = 1024;       // request descriptors in flight (ring entries)
constexpr int kServeMaxSlots = 1024;   // completion slots
constexpr int kServeHard = 0, kServeSoft = 1;

// One published request: copied into a device-memory ring entry before its
// items are published, never changed while any of its items is unfinished.
struct ServeDesc {
  long long seq;
  long long item_base;     // global index of the request's first work item
  int kind, n, k, W, H;
  int n_items;             // hard: tiles; soft: tile groups
  int slot;                // completion slot
  int ck, cap, pad0;
  float bg[3];
  float inv_tc, seed_scale, pad1;
  const float* packed;     // [n][kRec]
  float* out_rgb;          // [H][W][3] (soft: may be NULL)
  int* out_idx;            // hard: [H][W] or NULL
  const float* target;     // soft: [H][W][3]
  float* partial;          // soft: [n_items][n][8]
  double* loss_part;       // soft: [n_items]
  const float* probs;      // soft: [n][k]
  const float* palette;    // soft: [k][3]
  float* grad8;            // soft: [n][8]
  float* out_grad;         // soft: [5n + nk] (cx, cy, theta, length, half_width, logits)
  float* out_loss;         // soft: device scalar or NULL
  unsigned long long* status;  // [ST_COUNT]
  const volatile int* ready;   // NULL, or the word each item waits for (nonzero = go)
  unsigned long long ready_wait_ns;
};

// Control block in mapped pinned memory.
struct ServeCtl {
  volatile long long published;              // items published by the host
  volatile int stop;                         // host asks the kernel to exit
  volatile int pad;
  volatile long long done[kServeMaxSlots];   // seq of the last request completed in each slot
};

struct ServeArgs {
  ServeCtl* ctl;
  ServeDesc* ring;          // device memory [kServeRing]
  long long* next_item;    // device: items claimed
  int* items_done;         // device: per slot
  int* idle_ctas;          // device: CTAs currently without work (reset before each launch)
  int* closing;            // device: set once every CTA has been idle (reset before each launch)
  float4* rec;             // per-CTA scratch [grid][cap][256]
  int* rec_i;
  float4* ckpt;            // per-CTA scratch [grid][nck_max][256]
  float* ck_lt;
  int cap;
  size_t nck_max;
  long long first_seq;     // oldest request that may still have unclaimed items
  unsigned long long idle_ns;
  int grid;
};

int serve_grid();
cudaError_t launch_serve(const ServeArgs& a, cudaStream_t st);

}  // namespace tbr
