// Replay adjoint of the coupling variant Phi_g (Sec. "A variant closer to
// line-source potential flow", Eq. coupling; the replay of Sec. 5.2 with
// Eq. rpos, Eq. rT, Eq. adjstep, Eq. adjparam).  Per pixel, for i = 1..N:
//   x_i = Phi_g,i(x_{i-1}) in FP32 displacement form, or the side-table record
//   where the forward's floor bound, or the position checkpoint;
//   log T_i from the coverage of the deposit {u <= A_L(r) g(v)};
//   the adjoint step as the hand-derived reverse product of psi_g's
//   displacement and of the coverage (tbr_coupled_vjp.cuh).
// Two vertically adjacent pixels per thread on the persistent grid of 32x16
// tiles, in packed FP32 pairs (phi_pair_g, coupled_vjp2; tbr_pair.cuh), with
// the scalar routines for pops, checkpoints, flank-to-cap regeneration and
// direct-form steps; strokes streamed first to last through the shared-memory
// ring.  The 8 per-stroke gradient values go through the same warp
// reduce-scatter and CTA slice as the capsule map's adjoint, so the epilogue's
// fixed-order sum applies unchanged.
#include "tbr_pair.cuh"

namespace tbr {

namespace {

constexpr int kBwdCCH = 32;  // kBwdCCH * 8 == kTileThreads: one partial per thread per chunk

template <int CH>
__global__ void __launch_bounds__(kTileThreads, 2) k_backward_c2(BwdArgs a) {
  __shared__ __align__(128) float sbuf[2 * CH * kRec];
  __shared__ __align__(8) uint64_t sbar[2];
  __shared__ float red[2][kTileThreads / 32][CH * 8];
  __shared__ __align__(16) f2 pbuf[CH * kPairRec];
  __shared__ __align__(16) f2 gext[CH * kPairExtG];
  const int lane = threadIdx.x & 31;
  const int W = a.W, H = a.H, n = a.n;
  const int ntiles = pair_tile_count(W, H);
  const size_t P = static_cast<size_t>(W) * H;
  unsigned long long* status = a.status;
  const bool skip = status[ST_INVALID] != 0ull || status[ST_OVERFLOW] != 0ull;
  ChunkRing<CH> ring;
  ring.init(sbuf, sbar);
  float* slice = a.partial + static_cast<size_t>(blockIdx.x) * n * 8;
  unsigned drift = 0;
  bool first = true;
  RecordView rv{const_cast<float4*>(a.rec), const_cast<int*>(a.rec_i), const_cast<float4*>(a.ckpt),
                const_cast<float*>(a.ck_lt), P, 0, a.cap, a.ck_every};
  rv.drift_tol = a.drift_tol;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int px, py0;
    pair_tile_pixel(tile, W, px, py0);
    bool valid[2];
    size_t off[2];
    PixelState st[2];
    float lC[2][3];
    load_pair(a, px, py0, skip, valid, off, st, lC);
    if (!backward_tile2<CH, false, 1, true, true>(ring, a.packed, n, valid, st, lC, a.bg, rv, off, pbuf, red,
                                                  slice, first, drift, status, gext))
      break;
    first = false;
  }
  const unsigned dsum = __reduce_add_sync(0xffffffffu, drift);
  if (lane == 0 && dsum) atomicAdd(status + ST_DRIFT, static_cast<unsigned long long>(dsum));
}

}  // namespace

int backward_grid_coupled(int W, int H) {
  static PerDeviceInt cache;
  const int per_sm = cache.get([](int) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward_c2<kBwdCCH>, kTileThreads, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    return b;
  });
  const int tiles = pair_tile_count(W, H);
  const int g0 = per_sm * device_sm_count();
  const int waves = (tiles + g0 - 1) / g0;
  return (tiles + waves - 1) / waves;
}

cudaError_t launch_backward_coupled(const BwdArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  KernelTimer kt(TBR_K_BACKWARD, st);
  k_backward_c2<kBwdCCH><<<a.grid, kTileThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tbr
