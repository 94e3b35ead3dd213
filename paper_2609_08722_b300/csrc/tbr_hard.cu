// Hard render (Sec. 3, Eq. chain and Eq. render with alpha = indicator of the
// closed footprint K_i).  A CTA per 32x8 pixel tile, one live pixel per thread;
// the packed strokes stream through shared memory in chunks of CH records by
// 1-D bulk TMA (cp.async.bulk + mbarrier), last chunk first, and every thread
// reads the current stroke as a shared-memory broadcast.  After each chunk the
// pixels still in the chain are compacted onto the first threads
// (hard_tile_compact, tbr_tile.cuh), so finished pixels leave no idle lanes.
// The transfer renderer R_D keeps the capsule membership and replaces the
// transport by the sixteen-drop pull-back (drops_step); the coupling variant
// (Eq. coupling) replaces footprint and map by the deposit {u <= A_L(r) g(v)}
// and psi_g.
#include "tbr_tile.cuh"

namespace tbr {

namespace {

constexpr int kHardCH = 64;

template <int CH, bool DROPS, bool COUPLED>
__global__ void __launch_bounds__(kTileThreads) k_hard(const float* __restrict__ packed, int n, int W, int H,
                                                       float bg0, float bg1, float bg2,
                                                       float* __restrict__ out_rgb, int* __restrict__ out_idx,
                                                       unsigned long long* __restrict__ status, int want_stats) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  __shared__ HardLive live;
  const bool poison = status[ST_INVALID] != 0ull;
  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  const float bg[3] = {bg0, bg1, bg2};
  unsigned band = 0, visited = 0, background = 0;
  hard_tile_compact<CH, DROPS, COUPLED>(ring, packed, n, blockIdx.x, W, H, bg, poison, out_rgb, out_idx, live,
                                        band, visited, background, status);
  if (want_stats) {
    const unsigned bsum = __reduce_add_sync(0xffffffffu, band);
    const unsigned vsum = __reduce_add_sync(0xffffffffu, visited);
    const unsigned bgs = __reduce_add_sync(0xffffffffu, background);
    if ((threadIdx.x & 31) == 0) {
      if (bsum) atomicAdd(status + ST_BAND, static_cast<unsigned long long>(bsum));
      if (vsum) atomicAdd(status + ST_VISITED, static_cast<unsigned long long>(vsum));
      if (bgs) atomicAdd(status + ST_BG, static_cast<unsigned long long>(bgs));
    }
  }
}

}  // namespace

cudaError_t launch_hard(const float* packed, int n, int W, int H, const float bg[3], float* out_rgb,
                        int* out_idx, unsigned long long* status, int want_stats, cudaStream_t st, int transport) {
  const int tiles = tile_count(W, H);
  KernelTimer kt(TBR_K_HARD, st);
  if (transport == kTransportDrops)
    k_hard<kHardCH, true, false><<<tiles, kTileThreads, 0, st>>>(packed, n, W, H, bg[0], bg[1], bg[2], out_rgb,
                                                                 out_idx, status, want_stats);
  else if (transport == kTransportCoupled)
    k_hard<kHardCH, false, true><<<tiles, kTileThreads, 0, st>>>(packed, n, W, H, bg[0], bg[1], bg[2], out_rgb,
                                                                 out_idx, status, want_stats);
  else
    k_hard<kHardCH, false, false><<<tiles, kTileThreads, 0, st>>>(packed, n, W, H, bg[0], bg[1], bg[2], out_rgb,
                                                                  out_idx, status, want_stats);
  return cudaGetLastError();
}

}  // namespace tbr
