// lbm_wave.cuh -- the wavefront step of a batch of lattices: both passes of
// a time step (densities, Eq. A.4; forces, equilibrium, collision and
// streaming, Eqs. 1, 3-6, A.3) for several independent lattices in one
// persistent launch.
//
// Items are those of the single-lattice wavefront launch (k_wave: a tile of
// 32 x by nodes of one plane, group g = 0 .. nz + lag - 1, summing plane
// (g - 1) mod nz and colliding plane g - lag), numbered lattice by lattice
// and group-major inside a lattice, and the blocks of the grid take them from
// one atomic ticket.  A collision waits only on items of earlier groups of
// its own lattice, i.e. on smaller tickets, so the argument of k_wave holds
// unchanged: the block holding the smallest unfinished ticket waits on
// nothing unfinished and every wait ends.  Each lattice keeps its own flags
// and epoch in its own workspace; the ticket and the count of finished
// blocks live in the first lattice's.  Every lattice's L2 reuse distance is
// lag of its own planes, and small lattices that could not keep the GPU busy
// alone share one launch.  All lattices of a launch are at the same AA
// parity (a batch whose lattices differ takes one launch per parity).
#pragma once
#include "lbm_device.cuh"

namespace hmcsc {
namespace {

struct WaveLattice {
  StepParams p;
  Workspace w;
  int tp;           // tiles per plane: ntx * ceil(ny / by)
  unsigned first;   // first ticket of the lattice in the launch
};
struct WaveBatch {
  int n;               // lattices
  int lag;
  unsigned items;      // tickets of the launch
  unsigned spin_limit; // polls of one flag before a wait gives up
  long long hold;      // a flag of lattice 0 left unpublished (-1: none;
                       // failure-path tests)
  WaveLattice lat[kBatchMax];
};

// The block copies the parameters of the lattice its item belongs to into
// shared memory when that lattice changes (items come lattice by lattice,
// so rarely), and runs the item exactly as k_wave does.
template <int PARITY, int ST, bool PC, int CFG>
__global__ void __launch_bounds__(WaveShape<ST, CFG>::threads, WaveShape<ST, CFG>::minb)
    k_wave_batch(const __grid_constant__ WaveBatch b) {
  using T2 = typename Codec2<ST>::T2;
  constexpr int BY = WaveShape<ST, CFG>::c.by, NT = kTile * BY;
  extern __shared__ __align__(16) unsigned char wave_batch_smem[];
  T2(*buf)[kQ][NT] = reinterpret_cast<T2(*)[kQ][NT]>(wave_batch_smem);
  __shared__ unsigned s_ticket[2];
  __shared__ __align__(16) WaveLattice s_lat;
  __shared__ unsigned *s_ctls[kBatchMax];
  const int tid = threadIdx.y * kTile + threadIdx.x;
  unsigned *ctl0 = b.lat[0].w.wave;
  if (tid == 0) s_ticket[0] = atomicAdd(&ctl0[0], 1u);
  for (int l = tid; l < b.n; l += NT) s_ctls[l] = b.lat[l].w.wave;
  __syncthreads();
  unsigned k = s_ticket[0];
  int it = 0, cur = -1;
  unsigned epoch = 0;
  WaveArgs a{0u, 0, b.lag, b.spin_limit, -1};
  while (k < b.items) {
    it ^= 1;
    if (tid == 0) s_ticket[it] = atomicAdd(&ctl0[0], 1u);  // next item, read at the end
    int r = 0;
    {
      int lo = 0, hi = b.n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.lat[mid].first <= k) lo = mid; else hi = mid - 1;
      }
      r = lo;
    }
    if (r != cur) {     // block-uniform
      __syncthreads();  // the previous item's flag release has read s_lat
      const unsigned *src = reinterpret_cast<const unsigned *>(&b.lat[r]);
      unsigned *dst = reinterpret_cast<unsigned *>(&s_lat);
      for (int i = tid; i < (int)(sizeof(WaveLattice) / 4); i += NT) dst[i] = src[i];
      __syncthreads();
      epoch = *(volatile unsigned *)&s_lat.w.wave[2] + 1u;
      a.tp = s_lat.tp;
      a.hold = r == 0 ? b.hold : -1;
      cur = r;
    }
    wave_tile_item<PARITY, ST, PC, BY>(s_lat.p, s_lat.w, k - s_lat.first, a, a.hold, buf, epoch);
    k = s_ticket[it];
  }
  wave_exit(ctl0, s_ctls, b.n);
}

}  // namespace
}  // namespace hmcsc
