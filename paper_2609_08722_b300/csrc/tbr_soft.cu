// Soft forward render (Eq. relax, Eq. state) with the replay record of Sec. 5.2;
// forward-only instances for the sixteen-drop transport and the coupling
// variant (Eq. coupling: coverage sigmoid((sigma_b(v) - sigma') / w) and psi_g).
// One thread per pixel, a CTA per 32x8 tile, strokes streamed last-to-first
// through a two-deep shared-memory ring filled by 1-D bulk TMA.  Per stroke:
// distance sigma', coverage alpha = sigmoid(z) in logit form, compositing
// C += T alpha c, log2 T += log2(1 - alpha), then psi with the epsilon-floor.
// When recording: a sample the floor touched pushes (x_i, i) onto the pixel's
// side table (Lemma "Support of the replay record"), every k-th stroke stores
// (x_i, log2 T_i), and s_0 = (x_0, log2 T_0, record count) closes the pixel.
// One pixel per thread here.  A two-pixel form (soft_forward_tile2, as the
// serving kernel runs it) measured 5.99 vs 6.16 ms at 1024^2 x 2000, but its
// roundings match the adjoint's paired regeneration less closely: along a fit,
// a checkpoint then drifts past the tolerance every few steps, and the FP64
// repair of one such pixel (a serial replay of all its strokes) costs 5-13 ms.
#include <math.h>

#include "tbr_tile.cuh"

namespace tbr {

namespace {

constexpr int kSoftCH = 128;

template <int CH, bool RECORD, bool INERT, bool DROPS, bool COUPLED, bool EXIT>
__device__ __forceinline__ void soft_body(const SoftArgs& a) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  const int lane = threadIdx.x & 31;
  const int W = a.W, H = a.H;
  int px, py;
  tile_pixel(blockIdx.x, W, px, py);
  const bool valid = px < W && py < H;
  const size_t P = static_cast<size_t>(W) * H;
  const size_t p = valid ? static_cast<size_t>(py) * W + px : 0;
  unsigned long long* status = a.status;
  const bool invalid_prog = status[ST_INVALID] != 0ull;
  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  RecordView rv{a.rec, a.rec_i, a.ckpt, a.ck_lt, P, p, a.cap, a.ck_every};
  PixelState st;
  const bool ok = soft_forward_tile<CH, RECORD, INERT, DROPS, COUPLED, EXIT>(
      ring, a.packed, a.n, valid, (static_cast<float>(px) + 0.5f) / static_cast<float>(W),
      (static_cast<float>(py) + 0.5f) / static_cast<float>(H), rv, st, status, a.exit_lt);
  if (valid) {
    const float T0 = ex2_a(st.lt);
    float o0 = fmaf(T0, a.bg[0], st.C0), o1 = fmaf(T0, a.bg[1], st.C1), o2 = fmaf(T0, a.bg[2], st.C2);
    if (invalid_prog || !ok) o0 = o1 = o2 = __int_as_float(0x7fc00000);
    a.out_rgb[3 * p + 0] = o0;
    a.out_rgb[3 * p + 1] = o1;
    a.out_rgb[3 * p + 2] = o2;
    if (RECORD) {
      a.s0[p] = make_float4(st.xh, st.yh, st.xl, st.yl);
      a.s0b[p] = make_float2(st.lt, __int_as_float(st.cnt));
    }
  }
  if (RECORD) {
    const unsigned c = valid ? static_cast<unsigned>(st.cnt) : 0u;
    const unsigned tot = __reduce_add_sync(0xffffffffu, c);
    const unsigned mx = __reduce_max_sync(0xffffffffu, c);
    const unsigned ovf = __reduce_add_sync(0xffffffffu, (c > static_cast<unsigned>(a.cap)) ? 1u : 0u);
    if (lane == 0) {
      if (tot) atomicAdd(status + ST_RECORDS, static_cast<unsigned long long>(tot));
      if (mx) atomicMax(status + ST_MAXREC, static_cast<unsigned long long>(mx));
      if (ovf) atomicAdd(status + ST_OVERFLOW, static_cast<unsigned long long>(ovf));
    }
  }
}

template <int CH, bool RECORD, bool INERT, bool DROPS = false, bool COUPLED = false, bool EXIT = false>
__global__ void __launch_bounds__(kTileThreads) k_soft(SoftArgs a) {
  soft_body<CH, RECORD, INERT, DROPS, COUPLED, EXIT>(a);
}


}  // namespace

cudaError_t launch_soft(const SoftArgs& a, cudaStream_t st) {
  const int tiles = tile_count(a.W, a.H);
  const bool rec = a.s0 != nullptr;
  KernelTimer kt(TBR_K_SOFT, st);
  // forward-only renders that ask for the early exit run their own instances,
  // so the others carry no per-stroke test
  const bool ex = !rec && a.exit_lt > -1.0e38f;
  if (a.transport == kTransportDrops) {
    if (ex) k_soft<kSoftCH, false, false, true, false, true><<<tiles, kTileThreads, 0, st>>>(a);
    else k_soft<kSoftCH, false, false, true><<<tiles, kTileThreads, 0, st>>>(a);
  } else if (a.transport == kTransportCoupled) {
    if (rec) k_soft<kSoftCH, true, false, false, true><<<tiles, kTileThreads, 0, st>>>(a);
    else if (ex) k_soft<kSoftCH, false, false, false, true, true><<<tiles, kTileThreads, 0, st>>>(a);
    else k_soft<kSoftCH, false, false, false, true><<<tiles, kTileThreads, 0, st>>>(a);
  } else if (rec && a.inert) {
    k_soft<kSoftCH, true, true><<<tiles, kTileThreads, 0, st>>>(a);
  } else if (rec) {
    k_soft<kSoftCH, true, false><<<tiles, kTileThreads, 0, st>>>(a);
  } else if (a.inert) {
    if (ex) k_soft<kSoftCH, false, true, false, false, true><<<tiles, kTileThreads, 0, st>>>(a);
    else k_soft<kSoftCH, false, true><<<tiles, kTileThreads, 0, st>>>(a);
  } else {
    if (ex) k_soft<kSoftCH, false, false, false, false, true><<<tiles, kTileThreads, 0, st>>>(a);
    else k_soft<kSoftCH, false, false><<<tiles, kTileThreads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace tbr
