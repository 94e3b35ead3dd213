// Replay adjoint of the soft render (Sec. 5.2).  Per pixel, for i = 1..N:
//   x_i = Phi_i(x_{i-1})                   (Eq. rpos; Eq. fwd)
//         or the side-table record (i, x_i) where the forward's floor bound
//         (Lemma "Support of the replay record"),
//         or the position checkpoint every k strokes;
//   log T_i = log T_{i-1} - log(1 - alpha_i) (Eq. rT), or the checkpoint;
//   the adjoint step and the parameter gradients (Eq. adjstep, Eq. adjparam).
// The pixel-level work is one thread per pixel on a persistent grid; each CTA
// walks its tiles one after another, streaming the packed strokes first-to-last
// through a two-deep shared-memory ring (1-D bulk TMA).  The 8 per-stroke
// gradient values (cx, cy, theta, L, r, and the colour gradient) are reduced
// over the warp by a reduce-scatter of shuffles, over the CTA through shared
// memory, and written to the CTA's own slice of a partial buffer (no atomics);
// an epilogue sums the slices in a fixed order, so the result is reproducible.
#include <limits.h>
#include <math.h>

#include "tbr_pair.cuh"

namespace tbr {

namespace {

constexpr int kBwdCH = 32;  // kBwdCH * 8 == kTileThreads: one partial per thread per chunk

template <int CH, bool INERT>
__global__ void __launch_bounds__(kTileThreads, 4) k_backward(BwdArgs a) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  __shared__ float red[2][kTileThreads / 32][CH * 8];
  const int lane = threadIdx.x & 31;
  const int W = a.W, H = a.H, n = a.n;
  const int ntiles = ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
  const size_t P = static_cast<size_t>(W) * H;
  unsigned long long* status = a.status;
  const bool skip = status[ST_INVALID] != 0ull || status[ST_OVERFLOW] != 0ull;
  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  float* slice = a.partial + static_cast<size_t>(blockIdx.x) * n * 8;
  unsigned drift = 0;
  bool first = true;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int px, py;
    tile_pixel(tile, W, px, py);
    const bool valid = px < W && py < H && !skip;
    const size_t p = valid ? static_cast<size_t>(py) * W + px : 0;
    PixelState st{};
    float lC0 = 0.0f, lC1 = 0.0f, lC2 = 0.0f;
    if (valid) {
      const float4 s0 = a.s0[p];
      const float2 s0b = a.s0b[p];
      st.xh = s0.x; st.yh = s0.y; st.xl = s0.z; st.yl = s0.w;
      st.lt = s0b.x;
      st.cnt = __float_as_int(s0b.y);
      lC0 = a.dLdR[3 * p + 0]; lC1 = a.dLdR[3 * p + 1]; lC2 = a.dLdR[3 * p + 2];
    }
    RecordView rv{const_cast<float4*>(a.rec), const_cast<int*>(a.rec_i), const_cast<float4*>(a.ckpt),
                  const_cast<float*>(a.ck_lt), P, p, a.cap, a.ck_every};
    if (!backward_tile<CH, INERT>(ring, a.packed, n, valid, st, lC0, lC1, lC2, a.bg, rv, red, slice, first,
                                  drift, status))
      break;
    first = false;
  }
  const unsigned dsum = __reduce_add_sync(0xffffffffu, drift);
  if (lane == 0 && dsum) atomicAdd(status + ST_DRIFT, static_cast<unsigned long long>(dsum));
}

// The same replay adjoint with two vertically adjacent pixels per thread
// (32 x 16 tiles, packed FP32 pair arithmetic; tbr_pair.cuh).  Used for the
// exterior-transport model; the inert-mark model keeps k_backward.  The plain
// instance flags every tile in which a checkpoint drifted (a.tile_drift).  The
// QUEUE instance runs only when drift was counted, and then only over the
// flagged tiles: it repeats their computation (writing no slices) and queues
// each drifting pixel for the FP64 repair; otherwise it returns at once.
// Keeping the queue out of the plain instance keeps its hot loop free of that
// code.
template <int CH, bool QUEUE>
__global__ void __launch_bounds__(kTileThreads, 2) k_backward2(BwdArgs a) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  __shared__ float red[2][kTileThreads / 32][CH * 8];
  __shared__ __align__(16) f2 pbuf[CH * kPairRec];
  const int lane = threadIdx.x & 31;
  const int W = a.W, H = a.H, n = a.n;
  const int ntiles = ((W + kPairTileW - 1) / kPairTileW) * ((H + kPairTileH - 1) / kPairTileH);
  const size_t P = static_cast<size_t>(W) * H;
  unsigned long long* status = a.status;
  if (QUEUE && status[ST_DRIFT] == 0ull) return;
  const bool skip = status[ST_INVALID] != 0ull || status[ST_OVERFLOW] != 0ull;
  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  float* slice = a.partial + static_cast<size_t>(blockIdx.x) * n * 8;
  unsigned drift = 0;
  bool first = true;
  RecordView rv{const_cast<float4*>(a.rec), const_cast<int*>(a.rec_i), const_cast<float4*>(a.ckpt),
                const_cast<float*>(a.ck_lt), P, 0, a.cap, a.ck_every};
  rv.drift_tol = a.drift_tol;
  rv.repair_list = a.repair_list;
  rv.repair_count = a.repair_count;
  rv.repair_cap = a.repair_cap;
  rv.repair_first = a.repair_first;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (QUEUE && a.tile_drift[tile] == 0) continue;  // CTA-uniform
    int px, py0;
    pair_tile_pixel(tile, W, px, py0);
    bool valid[2];
    size_t off[2];
    PixelState st[2];
    float lC[2][3];
    load_pair(a, px, py0, skip, valid, off, st, lC);
    const unsigned drift0 = drift;
    // two strokes per loop iteration let the compiler overlap their independent work
    if (!backward_tile2<CH, QUEUE, 2, false, true>(ring, a.packed, n, valid, st, lC, a.bg, rv, off, pbuf, red,
                                                   slice, first, drift, status))
      break;
    if (!QUEUE && a.tile_drift && __syncthreads_or(drift != drift0) && threadIdx.x == 0) a.tile_drift[tile] = 1;
    first = false;
  }
  if (!QUEUE) {
    const unsigned dsum = __reduce_add_sync(0xffffffffu, drift);
    if (lane == 0 && dsum) atomicAdd(status + ST_DRIFT, static_cast<unsigned long long>(dsum));
  }
}

// Sorts the repair list by pixel index (one CTA, bitonic in shared memory) so
// that the repair and the correction sums run in a fixed order.  With more
// drifting pixels than the list holds, nothing is repaired and the count is
// reported instead.
__global__ void __launch_bounds__(kRepairMax) k_repair_sort(int2* list, const int* count, int cap,
                                                           unsigned long long* status) {
  __shared__ int2 sh[kRepairMax];
  const int c = *count;
  if (c > cap) {
    if (threadIdx.x == 0) atomicAdd(status + ST_REPAIR_OVF, static_cast<unsigned long long>(c));
    return;
  }
  int m = 1;
  while (m < c) m <<= 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) sh[i] = i < c ? list[i] : make_int2(INT_MAX, 0);
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const int2 u = sh[i], v = sh[l];
          if ((u.x > v.x) == up) { sh[i] = v; sh[l] = u; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < c; i += blockDim.x) list[i] = sh[i];
  if (threadIdx.x == 0 && c > 0) atomicAdd(status + ST_REPAIRED, static_cast<unsigned long long>(c));
}

// FP64 repair of a drifting checkpoint segment (the conditioning safeguard of
// Sec. 5.2): entry e replays its pixel's pair exactly as k_backward2 did (the
// main values), and from the start of the drifting segment on a second copy of
// the pixel whose positions are regenerated by Phi in FP64 -- side-table pops
// and checkpoint resets as in the main replay -- with coverage, adjoint step
// and VJP in FP32 at those positions.  It writes, per stroke, the repaired
// minus the main gradient values of the pixel; the epilogue adds them.
__global__ void __launch_bounds__(64) k_repair(BwdArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int count = *a.repair_count;
  if (count > a.repair_cap || e >= count) return;
  const int2 ent = a.repair_list[e];
  const int p = ent.x, seg = ent.y;
  const int W = a.W, n = a.n, ck = a.ck_every;
  const int px = p % W, py = p / W, py0 = py & ~1, ct = py & 1;
  const size_t P = static_cast<size_t>(W) * a.H;
  bool valid[2];
  size_t off[2];
  PixelState st[2];
  float lC[2][3];
  load_pair(a, px, py0, false, valid, off, st, lC);
  RecordView rv{const_cast<float4*>(a.rec), const_cast<int*>(a.rec_i), const_cast<float4*>(a.ckpt),
                const_cast<float*>(a.ck_lt), P, 0, a.cap, ck};
  rv.drift_tol = a.drift_tol;
  PairState ps;
  pair_state_init(ps, valid, st, lC, rv, off);
  PixAdj ra{};
  double x64 = 0.0, y64 = 0.0;
  bool active = false;
  auto start = [&]() {
    ra = PixAdj{comp(ps.Xh, ct), comp(ps.Yh, ct), comp(ps.Xl, ct), comp(ps.Yl, ct), comp(ps.LT, ct),
                comp(ps.LD, ct), comp(ps.LX, ct), comp(ps.LY, ct)};
    x64 = static_cast<double>(ra.xh) + static_cast<double>(ra.xl);
    y64 = static_cast<double>(ra.yh) + static_cast<double>(ra.yl);
    active = true;
  };
  if (seg == 0) start();
  float* out = a.corr + static_cast<size_t>(e) * n * 8;
  int next_ck = (ck < n) ? ck : 0;
  f2 Pr[kPairRec];
  for (int i1 = 1; i1 <= n; ++i1) {
    const float* S = a.packed + static_cast<size_t>(i1 - 1) * kRec;
#pragma unroll
    for (int k = 0; k < kPairRec; ++k) Pr[k] = F2(S[k]);
    // the colour step c_i - c_{i-1}, as the adjoint's pair records hold it (pair_records_fill)
#pragma unroll
    for (int c = 0; c < 3; ++c) Pr[P_CR + c] = F2(S[F_CR + c] - (i1 > 1 ? S[F_CR + c - kRec] : a.bg[c]));
    const bool at_ck = (i1 == next_ck);
    size_t cko = 0;
    if (at_ck) {
      next_ck = (next_ck + ck < n) ? next_ck + ck : 0;
      cko = static_cast<size_t>(i1 / ck - 1) * P;
    }
    // the repaired copy pops the same record as the main replay (read before it advances)
    const bool pop = i1 == ps.nri[ct];
    const float4 rp = pop ? rv.rec[static_cast<size_t>(ps.rc[ct] - 1) * P + off[ct]] : make_float4(0, 0, 0, 0);
    float g[2][8];
    unsigned drift = 0;
    pair_stroke<false>(ps, S, Pr, i1, at_ck, cko, (i1 & (kRenorm - 1)) == 0, rv, valid, off, g, drift);
    float* o = out + static_cast<size_t>(i1 - 1) * 8;
    if (active) {
      float4 ckp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      float ckl = 0.0f;
      if (at_ck) {
        ckp = rv.ckpt[cko + off[ct]];
        ckl = rv.ck_lt[cko + off[ct]];
      }
      ra.xh = static_cast<float>(x64); ra.xl = static_cast<float>(x64 - static_cast<double>(ra.xh));
      ra.yh = static_cast<float>(y64); ra.yl = static_cast<float>(y64 - static_cast<double>(ra.yh));
      float v[8];
      scalar_stroke(ra, load_stroke(S), Pr, lC[ct][0], lC[ct][1], lC[ct][2], pop, at_ck, true, rp, ckp, ckl,
                    a.drift_tol, v);
      if (pop) {
        x64 = static_cast<double>(rp.x) + static_cast<double>(rp.z);
        y64 = static_cast<double>(rp.y) + static_cast<double>(rp.w);
      } else if (at_ck) {
        x64 = static_cast<double>(ckp.x) + static_cast<double>(ckp.z);
        y64 = static_cast<double>(ckp.y) + static_cast<double>(ckp.w);
      } else {
        phi_f64(x64, y64, S);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = v[k] - g[ct][k];
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = 0.0f;
      if (i1 == seg) start();
    }
  }
}

// grad8[t] = sum over CTAs g (in order) of partial[g][t], then over the repair
// entries (in pixel order) of their corrections, carried in FP64.
__global__ void k_grad_sum(const float* __restrict__ partial, int G, int n8, const float* __restrict__ corr,
                           const int* __restrict__ repair_count, int repair_cap, float* __restrict__ grad8) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n8) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += static_cast<double>(partial[static_cast<size_t>(g) * n8 + t]);
  if (corr) {
    const int c = *repair_count;
    if (c <= repair_cap)
      for (int e = 0; e < c; ++e) s += static_cast<double>(corr[static_cast<size_t>(e) * n8 + t]);
  }
  grad8[t] = static_cast<float>(s);
}

// Per stroke: geometry gradients, and the colour chain rule
// dc_i/dz_iq = p_iq (Pal_q - c_i) / tau_c for the logits.  Pal_q - c_i is
// formed as sum_q' p_iq' (Pal_q - Pal_q') (the weights sum to one): for the
// dominant entry it is a small difference of two nearly equal colours, which
// Pal_q - c_i would take from the rounding of c_i.  A drop (L = 0) without a
// coupling profile has no direction, so its angle gradient is exactly zero
// (the renders are invariant under theta there); the sums over pixels would
// only leave rounding.  A coupled drop's profile turns with theta.
__global__ void k_grad_out(EpilogueArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const bool bad = a.status[ST_INVALID] != 0ull || a.status[ST_OVERFLOW] != 0ull ||
                   a.status[ST_TIMEOUT] != 0ull;
  const float nan = __int_as_float(0x7fc00000);
  const float* g8 = a.grad8 + static_cast<size_t>(i) * 8;
  const float* R = a.packed + static_cast<size_t>(i) * kRec;
  a.g_cx[i] = bad ? nan : g8[0];
  a.g_cy[i] = bad ? nan : g8[1];
  const bool round_drop = R[F_L] == 0.0f && R[F_C1] == 0.0f && R[F_C1 + 1] == 0.0f && R[F_C1 + 2] == 0.0f;
  a.g_th[i] = bad ? nan : (round_drop ? 0.0f : g8[2]);
  a.g_len[i] = bad ? nan : g8[3];
  a.g_r[i] = bad ? nan : g8[4];
  const float* p = a.probs + static_cast<size_t>(i) * a.k;
  for (int q = 0; q < a.k; ++q) {
    const float* pal = a.palette + 3 * q;
    float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f;
    for (int u = 0; u < a.k; ++u) {
      const float* pu = a.palette + 3 * u;
      d0 = fmaf(p[u], pal[0] - pu[0], d0);
      d1 = fmaf(p[u], pal[1] - pu[1], d1);
      d2 = fmaf(p[u], pal[2] - pu[2], d2);
    }
    const float d = fmaf(d0, g8[5], fmaf(d1, g8[6], d2 * g8[7]));
    a.g_logits[static_cast<size_t>(i) * a.k + q] = bad ? nan : p[q] * d * a.inv_color_temp;
  }
}

// dL/dPal_q[c] = sum_i p_iq dL/dc_i[c]; one block per (q, c), FP64 block sum.
__global__ void k_grad_palette(EpilogueArgs a) {
  const int qc = blockIdx.x;
  const int q = qc / 3, c = qc % 3;
  double s = 0.0;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x)
    s += static_cast<double>(a.probs[static_cast<size_t>(i) * a.k + q]) *
         static_cast<double>(a.grad8[static_cast<size_t>(i) * 8 + 5 + c]);
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const bool bad = a.status[ST_INVALID] != 0ull || a.status[ST_OVERFLOW] != 0ull ||
                     a.status[ST_TIMEOUT] != 0ull;
    a.g_pal[qc] = bad ? __int_as_float(0x7fc00000) : static_cast<float>(sh[0]);
  }
}

}  // namespace

int device_sm_count() {
  static PerDeviceInt cache;
  return cache.get([](int dev) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    return sms;
  });
}

int backward_grid(int W, int H, int inert) {
  static PerDeviceInt pair_cache, one_cache;
  const int per_sm = inert ? one_cache.get([](int) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward<kBwdCH, true>, kTileThreads, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    return b;
  })
                           : pair_cache.get([](int) {
                               int b = 0;
                               if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward2<kBwdCH, false>,
                                                                                 kTileThreads, 0) != cudaSuccess ||
                                   b < 1)
                                 b = 1;
                               return b;
                             });
  const int tiles = inert ? ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH)
                          : ((W + kPairTileW - 1) / kPairTileW) * ((H + kPairTileH - 1) / kPairTileH);
  const int g0 = per_sm * device_sm_count();
  const int waves = (tiles + g0 - 1) / g0;
  return (tiles + waves - 1) / waves;
}

cudaError_t launch_backward(const BwdArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  if (a.coupled) return launch_backward_coupled(a, st);
  const bool repair = !a.inert && a.repair_list && a.repair_cap > 0;
  if (repair) {
    // repair_first holds the per-pixel queued flags, then the per-tile drift flags
    cudaError_t e = cudaMemsetAsync(a.repair_count, 0, sizeof(int), st);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(a.repair_first, 0, static_cast<size_t>(a.W) * a.H + pair_tile_count(a.W, a.H), st);
    if (e != cudaSuccess) return e;
  }
  {
    KernelTimer kt(TBR_K_BACKWARD, st);
    if (a.inert) k_backward<kBwdCH, true><<<a.grid, kTileThreads, 0, st>>>(a);
    else k_backward2<kBwdCH, false><<<a.grid, kTileThreads, 0, st>>>(a);
  }
  if (repair) {
    k_backward2<kBwdCH, true><<<a.grid, kTileThreads, 0, st>>>(a);  // returns at once without drift
    k_repair_sort<<<1, kRepairMax, 0, st>>>(a.repair_list, a.repair_count, a.repair_cap, a.status);
    k_repair<<<(a.repair_cap + 63) / 64, 64, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_backward_epilogue(const EpilogueArgs& a, cudaStream_t st) {
  if (a.n <= 0) {
    return cudaSuccess;
  }
  const int n8 = a.n * 8;
  KernelTimer kt(TBR_K_EPILOGUE, st);
  k_grad_sum<<<(n8 + 255) / 256, 256, 0, st>>>(a.partial, a.grid, n8, a.corr, a.repair_count, a.repair_cap,
                                               a.grad8);
  k_grad_out<<<(a.n + 127) / 128, 128, 0, st>>>(a);
  if (a.g_pal) k_grad_palette<<<a.k * 3, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tbr
