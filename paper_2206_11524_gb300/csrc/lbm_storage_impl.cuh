// lbm_storage_impl.cuh -- launchers of the storage-typed kernels for one
// storage kind.  Included once per kind by lbm_st_*.cu with HMCSC_ST (a
// StorageKind) and HMCSC_SUF (the name suffix) defined.
#include <mutex>

#include "lbm_wave.cuh"

#define HMCSC_CAT2(a, b) a##_##b
#define HMCSC_CAT(a, b) HMCSC_CAT2(a, b)
#define HMCSC_NAME(n) HMCSC_CAT(n, HMCSC_SUF)

namespace hmcsc {
namespace {
constexpr int kST = HMCSC_ST;

template <int PARITY, int CFG>
void density_cfg(const StepParams &p, const Workspace &w, cudaStream_t s) {
  constexpr Shape S = DensityShape<CFG>::s;
  const dim3 grid(p.ntx, (p.ny + S.by - 1) / S.by, (p.nz + S.bz - 1) / S.bz);
  k_density<PARITY, kST, CFG><<<grid, dim3(kTile, S.by, S.bz), 0, s>>>(p, w);
}
template <int PARITY, int CFG>
void collide_cfg(const StepParams &p, const Workspace &w, cudaStream_t s) {
  constexpr Shape S = CollideShape<PARITY, kST, CFG>::s;
  const dim3 grid(p.ntx, (p.ny + S.by - 1) / S.by, (p.nz + S.bz - 1) / S.bz);
  if (w.ns2)
    k_collide_stream<PARITY, kST, CFG, true><<<grid, dim3(kTile, S.by, S.bz), 0, s>>>(p, w);
  else
    k_collide_stream<PARITY, kST, CFG, false><<<grid, dim3(kTile, S.by, S.bz), 0, s>>>(p, w);
}
template <int PARITY>
void density_any(const StepParams &p, const Workspace &w, int cfg, cudaStream_t s) {
  switch (cfg) {
    case 1: density_cfg<PARITY, 1>(p, w, s); break;
    case 2: density_cfg<PARITY, 2>(p, w, s); break;
    default: density_cfg<PARITY, 0>(p, w, s);
  }
}
template <int PARITY, bool PC, int CFG>
void collide_pipe_launch(const StepParams &p, const Workspace &w, cudaStream_t s) {
  using T2 = typename Codec2<kST>::T2;
  constexpr Shape S = CollideShape<PARITY, kST, CFG>::s;
  constexpr PipeCfg P = pipe_cfg(CFG);
  constexpr int smem = pipe_smem_bytes(CFG, (int)sizeof(T2), PC);
  // the shared-memory limit is an attribute of the function on each device;
  // if setting it fails, the launch below reports the error
  static std::once_flag attr_once[16];
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 16)
    std::call_once(attr_once[dev], [] {
      cudaFuncSetAttribute(k_collide_pipe<PARITY, kST, PC, CFG>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
  const dim3 grid(p.ntx, (p.ny + S.by - 1) / S.by, (p.nz + P.zc - 1) / P.zc);
  k_collide_pipe<PARITY, kST, PC, CFG><<<grid, dim3(kTile, S.by, 1), smem, s>>>(p, w);
}
template <int PARITY, int CFG>
void collide_pipe_cfg(const StepParams &p, const Workspace &w, cudaStream_t s) {
  if (w.ns2)
    collide_pipe_launch<PARITY, true, CFG>(p, w, s);
  else
    collide_pipe_launch<PARITY, false, CFG>(p, w, s);
}
template <int PARITY>
void collide_any(const StepParams &p, const Workspace &w, int cfg, cudaStream_t s) {
  switch (cfg) {
    case 1: collide_cfg<PARITY, 1>(p, w, s); break;
    case 2: collide_cfg<PARITY, 2>(p, w, s); break;
    case 3: collide_cfg<PARITY, 3>(p, w, s); break;
    case 4: collide_cfg<PARITY, 4>(p, w, s); break;
    case 5: collide_pipe_cfg<PARITY, 5>(p, w, s); break;
    case 6: collide_pipe_cfg<PARITY, 6>(p, w, s); break;
    case 7: collide_pipe_cfg<PARITY, 7>(p, w, s); break;
    case 8: collide_pipe_cfg<PARITY, 8>(p, w, s); break;
    case 9: collide_pipe_cfg<PARITY, 9>(p, w, s); break;
    default: collide_cfg<PARITY, 0>(p, w, s);
  }
}
}  // namespace

cudaError_t HMCSC_NAME(launch_density)(const StepParams &p, const Workspace &w,
                                       int parity, int cfg, cudaStream_t s) {
  if (parity == 0) density_any<0>(p, w, cfg, s); else density_any<1>(p, w, cfg, s);
  return cudaGetLastError();
}

cudaError_t HMCSC_NAME(launch_collide)(const StepParams &p, const Workspace &w,
                                       int parity, int cfg, cudaStream_t s) {
  if (parity == 0) collide_any<0>(p, w, cfg, s); else collide_any<1>(p, w, cfg, s);
  return cudaGetLastError();
}

cudaError_t HMCSC_NAME(launch_fields)(const StepParams &p, const Workspace &w,
                                      int parity, cudaStream_t s) {
  const dim3 grid(p.ntx, (p.ny + kFieldsBY - 1) / kFieldsBY,
                  (p.nz + kFieldsBZ - 1) / kFieldsBZ);
  const dim3 block(kTile, kFieldsBY, kFieldsBZ);
  if (w.ns2) {
    if (parity == 0) k_fields<0, kST, true><<<grid, block, 0, s>>>(p, w);
    else k_fields<1, kST, true><<<grid, block, 0, s>>>(p, w);
  } else {
    if (parity == 0) k_fields<0, kST, false><<<grid, block, 0, s>>>(p, w);
    else k_fields<1, kST, false><<<grid, block, 0, s>>>(p, w);
  }
  return cudaGetLastError();
}

cudaError_t HMCSC_NAME(launch_init)(const StepParams &p, const Workspace &w,
                                    const float *rho_a, const float *rho_b,
                                    cudaStream_t s) {
  const long long N = (long long)p.nx * p.ny * p.nz;
  long long b = (N + 255) / 256;
  b = b < 1 ? 1 : (b > 4864 ? 4864 : b);
  k_init_equilibrium<kST><<<(unsigned)b, 256, 0, s>>>(p, w, rho_a, rho_b);
  return cudaGetLastError();
}

namespace {
template <int PARITY, bool PC>
cudaError_t single_pass(const StepParams &p, const Workspace &w, int nzc, cudaStream_t s) {
  const int ncol = p.ntx * kTile;
  const size_t smem = sp_ring_bytes(ncol);
  static bool attr_set = false;  // the largest ring any lattice may need
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_sp_bulk<PARITY, kST, PC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sp_ring_bytes(kSpMaxThreads));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int nyb = (p.ny + kSpBY - 1) / kSpBY;
  k_sp_bulk<PARITY, kST, PC><<<dim3(nyb, nzc), ncol, smem, s>>>(p, w, nzc);
  k_sp_seams<PARITY, kST, PC><<<dim3(p.ntx, nyb, (p.nz + 3) / 4), dim3(kTile, 4), 0, s>>>(p, w, nzc, 0);
  k_sp_seams<PARITY, kST, PC><<<dim3(p.ntx, (p.ny + 3) / 4, nzc), dim3(kTile, 4), 0, s>>>(p, w, nzc, 1);
  return cudaGetLastError();
}
}  // namespace

cudaError_t HMCSC_NAME(launch_single_pass)(const StepParams &p, const Workspace &w,
                                           int parity, int nzc, cudaStream_t s) {
  if (w.ns2)
    return parity == 0 ? single_pass<0, true>(p, w, nzc, s) : single_pass<1, true>(p, w, nzc, s);
  return parity == 0 ? single_pass<0, false>(p, w, nzc, s) : single_pass<1, false>(p, w, nzc, s);
}

namespace {
// Resident blocks per SM and SM count of the current device for one k_wave
// instance (the grid is one wave of persistent blocks).
struct WaveOccupancy {
  int dev = -1, per_sm = 0, sms = 0, l2 = 0;
};
template <int PARITY, bool PC, int CFG>
cudaError_t wave_launch(const StepParams &p, const Workspace &w, int lag, unsigned spin_limit,
                        long long hold, cudaStream_t s) {
  using T2 = typename Codec2<kST>::T2;
  constexpr int BY = wave_cfg(CFG).by, NT = kTile * BY;
  constexpr int smem = 2 * kQ * NT * (int)sizeof(T2);
  auto kern = k_wave<PARITY, kST, PC, CFG>;
  static WaveOccupancy occ[16];
  static std::mutex occ_mu;  // host threads may launch on a device first at once
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  std::unique_lock<std::mutex> lock(occ_mu);
  WaveOccupancy &o = occ[dev];
  if (o.dev != dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, kern, NT, smem);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (o.per_sm < 1) return cudaErrorInvalidConfiguration;
    o.dev = dev;
  }
  const int per_sm = o.per_sm, sms = o.sms;
  lock.unlock();
  WaveArgs a;
  a.tp = p.ntx * ((p.ny + BY - 1) / BY);
  a.lag = lag;
  a.items = (unsigned)((long long)(p.nz + lag) * a.tp);
  a.spin_limit = spin_limit;
  a.hold = hold;
  const long long want = (long long)per_sm * sms;
  const unsigned grid = (unsigned)(want < (long long)a.items ? want : (long long)a.items);
  // A cooperative launch: every block is resident while the others run.
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kTile, BY, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p, w, a);
}
template <int PARITY, int CFG>
cudaError_t wave_pc(const StepParams &p, const Workspace &w, int lag, unsigned spin,
                    long long hold, cudaStream_t s) {
  return w.ns2 ? wave_launch<PARITY, true, CFG>(p, w, lag, spin, hold, s)
               : wave_launch<PARITY, false, CFG>(p, w, lag, spin, hold, s);
}
template <int PARITY>
cudaError_t wave_any(const StepParams &p, const Workspace &w, int cfg, int lag, unsigned spin,
                     long long hold, cudaStream_t s) {
  switch (cfg) {
    case 2: return wave_pc<PARITY, 2>(p, w, lag, spin, hold, s);
    case 3: return wave_pc<PARITY, 3>(p, w, lag, spin, hold, s);
    default: return wave_pc<PARITY, 1>(p, w, lag, spin, hold, s);
  }
}
}  // namespace

cudaError_t HMCSC_NAME(launch_wave)(const StepParams &p, const Workspace &w, int parity,
                                    int cfg, int lag, unsigned spin_limit, long long hold,
                                    cudaStream_t s) {
  if (lag < kWaveLagMin) return cudaErrorInvalidValue;
  return parity == 0 ? wave_any<0>(p, w, cfg, lag, spin_limit, hold, s)
                     : wave_any<1>(p, w, cfg, lag, spin_limit, hold, s);
}

namespace {
// One persistent launch over the job's lattices idx[0..n) (all of AA parity
// PARITY), tiles of the wavefront shape CFG.
template <int PARITY, bool PC, int CFG>
cudaError_t wave_batch_launch(const WaveJob &job, const int *idx, int n, cudaStream_t s) {
  using T2 = typename Codec2<kST>::T2;
  constexpr int BY = wave_cfg(CFG).by, NT = kTile * BY;
  constexpr int smem = 2 * kQ * NT * (int)sizeof(T2);
  auto kern = k_wave_batch<PARITY, kST, PC, CFG>;
  static WaveOccupancy occ[16];
  static std::mutex occ_mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  std::unique_lock<std::mutex> lock(occ_mu);
  WaveOccupancy &o = occ[dev];
  if (o.dev != dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, kern, NT, smem);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&o.l2, cudaDevAttrL2CacheSize, dev);
    if (e != cudaSuccess) return e;
    if (o.per_sm < 1) return cudaErrorInvalidConfiguration;
    o.dev = dev;
  }
  const long long want = (long long)o.per_sm * o.sms;
  // a set's planes in flight may fill this much of L2
  const double set_budget = kWaveSetL2Share * o.l2;
  lock.unlock();
  static thread_local WaveBatch b;  // ~24 KB: kept off the stack
  // lattices by group count, most first (stable: equal counts keep the
  // job's order)
  int ord[kBatchMax];
  for (int k = 0; k < n; ++k) {
    int j = k;
    while (j > 0 && job.sp[idx[ord[j - 1]]]->nz < job.sp[idx[k]]->nz) {
      ord[j] = ord[j - 1];
      --j;
    }
    ord[j] = k;
  }
  b.n = n;
  b.lag = job.lag;
  b.spin_limit = job.spin_limit;
  b.hold_lat = -1;
  b.hold = job.hold;
  b.tsum[0] = 0;
  for (int k = 0; k < n; ++k) {
    WaveLattice &L = b.lat[k];
    L.p = *job.sp[idx[ord[k]]];
    L.w = *job.ws[idx[ord[k]]];
    L.tp = L.p.ntx * ((L.p.ny + BY - 1) / BY);
    b.tsum[k + 1] = b.tsum[k] + (unsigned)L.tp;
    if (idx[ord[k]] == 0) b.hold_lat = k;  // the withheld flag is the job's lattice 0's
  }
  // sets: runs of the order whose planes in flight fit the budget together
  // (a lattice alone may exceed it); segments inside a set: groups
  // [G_m, G_(m-1)) hold the set's lattices 0 .. m - 1
  unsigned long long first = 0;
  int nseg = 0;
  for (int lb = 0; lb < n;) {
    double bytes = 0.0;
    int le = lb;
    while (le < n) {
      const WaveLattice &L = b.lat[le];
      const double lat_bytes =
          (double)(job.lag + 2) * L.p.ntx * kTile * L.p.ny * kQ * (double)sizeof(T2);
      if (le > lb && bytes + lat_bytes > set_budget) break;
      bytes += lat_bytes;
      ++le;
    }
    int g0 = 0;
    for (int m = le - lb; m >= 1; --m) {
      const int gend = b.lat[lb + m - 1].p.nz + job.lag;
      if (gend <= g0) continue;
      b.seg_first[nseg] = (unsigned)first;
      b.seg_g0[nseg] = g0;
      b.seg_lb[nseg] = lb;
      b.seg_m[nseg] = m;
      first += (unsigned long long)(gend - g0) * (b.tsum[lb + m] - b.tsum[lb]);
      g0 = gend;
      ++nseg;
    }
    lb = le;
  }
  if (first > 0xFFFFFFFFull) return cudaErrorInvalidValue;  // the host checks this first
  b.nseg = nseg;
  b.items = (unsigned)first;
  const unsigned grid = (unsigned)(want < (long long)first ? want : (long long)first);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kTile, BY, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, b);
}
// Lattices of each parity in one launch each (a step of a batch whose
// lattices differ in parity is two launches in a row).
template <bool PC, int CFG>
cudaError_t wave_batch_parities(const WaveJob &job, cudaStream_t s) {
  int idx[2][kBatchMax], n[2] = {0, 0};
  for (int k = 0; k < job.n; ++k) {
    const int par = job.parity[k] & 1;
    idx[par][n[par]++] = k;
  }
  for (int par = 0; par < 2; ++par) {
    if (n[par] == 0) continue;
    const cudaError_t e = par == 0 ? wave_batch_launch<0, PC, CFG>(job, idx[0], n[0], s)
                                   : wave_batch_launch<1, PC, CFG>(job, idx[1], n[1], s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
template <int CFG>
cudaError_t wave_batch_pc(const WaveJob &job, cudaStream_t s) {
  return job.ws[0]->ns2 != nullptr ? wave_batch_parities<true, CFG>(job, s)
                                   : wave_batch_parities<false, CFG>(job, s);
}
}  // namespace

cudaError_t HMCSC_NAME(launch_wave_batch)(const WaveJob &job, cudaStream_t s) {
  if (job.n < 1 || job.n > kBatchMax || job.lag < kWaveLagMin) return cudaErrorInvalidValue;
  switch (job.cfg) {
    case 2: return wave_batch_pc<2>(job, s);
    case 3: return wave_batch_pc<3>(job, s);
    default: return wave_batch_pc<1>(job, s);
  }
}

cudaError_t HMCSC_NAME(launch_batch_density)(const BatchArgs &a, cudaStream_t s) {
  k_batch_density<kST><<<(unsigned)a.prefix[a.n], dim3(kTile, kBatchBY, 1), 0, s>>>(a);
  return cudaGetLastError();
}

namespace {
// k_batch_collide_pipe over the items of `a` at AA parity PARITY, shape CFG.
template <int PARITY, bool PC, int CFG>
cudaError_t batch_pipe_launch(const BatchArgs &a, cudaStream_t s) {
  using T2 = typename Codec2<kST>::T2;
  constexpr Shape S = CollideShape<PARITY, kST, CFG>::s;
  constexpr PipeCfg P = pipe_cfg(CFG);
  constexpr int smem = pipe_smem_bytes(CFG, (int)sizeof(T2), PC);
  static thread_local BatchArgs b;  // ~16 KB: kept off the stack
  b.n = 0;
  b.prefix[0] = 0;
  for (int k = 0; k < a.n; ++k) {
    if ((a.item[k].parity & 1) != PARITY) continue;
    BatchItem &it = b.item[b.n];
    it = a.item[k];
    it.gx = it.p.ntx;
    it.gy = (it.p.ny + S.by - 1) / S.by;
    const long long blocks =
        (long long)b.prefix[b.n] + (long long)it.gx * it.gy * ((it.p.nz + P.zc - 1) / P.zc);
    if (blocks > 2147483647LL) return cudaErrorInvalidValue;
    b.prefix[b.n + 1] = (int)blocks;
    ++b.n;
  }
  if (b.n == 0) return cudaSuccess;
  // the shared-memory limit is an attribute of the function on each device
  static std::once_flag attr_once[16];
  static cudaError_t attr_err[16];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  std::call_once(attr_once[dev], [dev] {
    attr_err[dev] = cudaFuncSetAttribute(k_batch_collide_pipe<PARITY, kST, PC, CFG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  if (attr_err[dev] != cudaSuccess) return attr_err[dev];
  k_batch_collide_pipe<PARITY, kST, PC, CFG>
      <<<(unsigned)b.prefix[b.n], dim3(kTile, S.by, 1), smem, s>>>(b);
  return cudaGetLastError();
}
template <int PARITY, bool PC>
cudaError_t batch_pipe_any(const BatchArgs &a, int cfg, cudaStream_t s) {
  switch (cfg) {
    case 5: return batch_pipe_launch<PARITY, PC, 5>(a, s);
    case 6: return batch_pipe_launch<PARITY, PC, 6>(a, s);
    case 7: return batch_pipe_launch<PARITY, PC, 7>(a, s);
    case 8: return batch_pipe_launch<PARITY, PC, 8>(a, s);
    case 9: return batch_pipe_launch<PARITY, PC, 9>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t HMCSC_NAME(launch_batch_collide_pipe)(const BatchArgs &a, int even_cfg, int odd_cfg,
                                                  cudaStream_t s) {
  const bool pc = a.item[0].w.ns2 != nullptr;
  cudaError_t e = pc ? batch_pipe_any<0, true>(a, even_cfg, s)
                     : batch_pipe_any<0, false>(a, even_cfg, s);
  if (e != cudaSuccess) return e;
  return pc ? batch_pipe_any<1, true>(a, odd_cfg, s) : batch_pipe_any<1, false>(a, odd_cfg, s);
}

cudaError_t HMCSC_NAME(launch_batch_collide)(const BatchArgs &a, cudaStream_t s) {
  const dim3 grid((unsigned)a.prefix[a.n]), block(kTile, kBatchBY, 1);
  if (a.item[0].w.ns2)
    k_batch_collide<kST, true><<<grid, block, 0, s>>>(a);
  else
    k_batch_collide<kST, false><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hmcsc
