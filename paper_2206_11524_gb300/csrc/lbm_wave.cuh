// lbm_wave.cuh -- the wavefront step of a batch of lattices: both passes of
// a time step (densities, Eq. A.4; forces, equilibrium, collision and
// streaming, Eqs. 1, 3-6, A.3) for several independent lattices in one
// persistent launch.
//
// Items are those of the single-lattice wavefront launch (k_wave: a tile of
// 32 x by nodes of one plane, group g = 0 .. nz + lag - 1, summing plane
// (g - 1) mod nz and colliding plane g - lag), numbered group-major across a
// set of lattices: group g of every lattice of the set that has one comes
// before group g + 1 of any (sets below).  The blocks of the grid take items
// from one atomic ticket.  A collision waits only on items of earlier
// groups of its own lattice, i.e. on smaller tickets, so the argument of
// k_wave holds unchanged: the block holding the smallest unfinished ticket
// waits on nothing unfinished and every wait ends.  Lattices of one set run
// side by side, so the chain of dependent groups is that of the set's
// deepest lattice, not the sum over the set: small lattices whose own chain
// could not keep the GPU busy fill it together.  Each lattice keeps its own
// flags and epoch in its own workspace; the ticket and the count of finished
// blocks live in the first lattice's.  All lattices of a launch are at the
// same AA parity (a batch whose lattices differ takes one launch per
// parity).
//
// Numbering.  The host orders the lattices by group count, most first, and
// cuts that order into sets whose planes in flight (lag + 2 planes of
// populations each) fit a share of L2 together, so the populations a
// density pass reads are still in L2 when the collision reads them.  Sets
// run one after another.  Inside a set of lattices with group counts G_0 >=
// G_1 >= ..., groups [G_m, G_(m-1)) (G_n = 0) hold exactly its lattices
// 0 .. m - 1: a segment of (G_(m-1) - G_m) groups of (tiles per plane of
// those m lattices) items each, in lattice order inside a group.
#pragma once
#include "lbm_device.cuh"

namespace hmcsc {
namespace {

struct WaveLattice {
  StepParams p;
  Workspace w;
  int tp;           // tiles per plane: ntx * ceil(ny / by)
};
struct WaveBatch {
  int n;               // lattices, most groups first
  int lag;
  int nseg;            // segments: runs of groups with the same lattices
  unsigned items;      // tickets of the launch
  unsigned spin_limit; // polls of one flag before a wait gives up
  int hold_lat;        // lattice whose flag `hold` is left unpublished
  long long hold;      // (-1: none; failure-path tests)
  unsigned seg_first[kBatchMax];  // first ticket of segment s
  int seg_g0[kBatchMax];          // its first group
  int seg_lb[kBatchMax];          // its lattices: seg_lb .. seg_lb + seg_m - 1
  int seg_m[kBatchMax];
  unsigned tsum[kBatchMax + 1];   // tsum[r] = tiles per plane of lattices < r
  WaveLattice lat[kBatchMax];
};
static_assert(sizeof(WaveBatch) <= 32000, "kernel parameter limit");

// Lattice r and its own item number (g * tp_r + tile) of ticket k.
__device__ __forceinline__ void wave_batch_item(const WaveBatch &b, unsigned k, int &r,
                                                unsigned &local) {
  int lo = 0, hi = b.nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.seg_first[mid] <= k) lo = mid; else hi = mid - 1;
  }
  const int lb = b.seg_lb[lo];
  const unsigned base = b.tsum[lb];
  const unsigned off = k - b.seg_first[lo], per = b.tsum[lb + b.seg_m[lo]] - base;
  const unsigned gg = off / per, rem = off - gg * per + base;
  const unsigned g = (unsigned)b.seg_g0[lo] + gg;
  int l = lb, h = lb + b.seg_m[lo] - 1;
  while (l < h) {
    const int mid = (l + h + 1) >> 1;
    if (b.tsum[mid] <= rem) l = mid; else h = mid - 1;
  }
  r = l;
  local = g * (unsigned)b.lat[l].tp + (rem - b.tsum[l]);
}

// The block runs each item exactly as k_wave does, reading the lattice's
// parameters from the launch's parameter block (the lattice changes from
// item to item, and a block-uniform constant load costs less than a copy).
template <int PARITY, int ST, bool PC, int CFG>
__global__ void __launch_bounds__(WaveShape<ST, CFG>::threads, WaveShape<ST, CFG>::minb)
    k_wave_batch(const __grid_constant__ WaveBatch b) {
  using T2 = typename Codec2<ST>::T2;
  constexpr int BY = WaveShape<ST, CFG>::c.by, NT = kTile * BY;
  extern __shared__ __align__(16) unsigned char wave_batch_smem[];
  T2(*buf)[kQ][NT] = reinterpret_cast<T2(*)[kQ][NT]>(wave_batch_smem);
  __shared__ unsigned s_ticket[2];
  __shared__ unsigned s_epoch[kBatchMax];
  __shared__ unsigned *s_ctls[kBatchMax];
  const int tid = threadIdx.y * kTile + threadIdx.x;
  unsigned *ctl0 = b.lat[0].w.wave;
  if (tid == 0) s_ticket[0] = atomicAdd(&ctl0[0], 1u);
  for (int l = tid; l < b.n; l += NT) {
    s_ctls[l] = b.lat[l].w.wave;
    s_epoch[l] = *(volatile unsigned *)&b.lat[l].w.wave[2] + 1u;
  }
  __syncthreads();
  unsigned k = s_ticket[0];
  int it = 0;
  while (k < b.items) {
    it ^= 1;
    if (tid == 0) s_ticket[it] = atomicAdd(&ctl0[0], 1u);  // next item, read at the end
    int r;
    unsigned local;
    wave_batch_item(b, k, r, local);
    const WaveLattice &L = b.lat[r];
    const long long hold = r == b.hold_lat ? b.hold : -1;
    const WaveArgs a{0u, L.tp, b.lag, b.spin_limit, hold};
    wave_tile_item<PARITY, ST, PC, BY>(L.p, L.w, local, a, hold, buf, s_epoch[r]);
    k = s_ticket[it];
  }
  wave_exit(ctl0, s_ctls, b.n);
}

}  // namespace
}  // namespace hmcsc
