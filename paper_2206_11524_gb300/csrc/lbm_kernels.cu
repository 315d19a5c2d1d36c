// lbm_kernels.cu -- storage-independent kernels (geometry, observables)
// and the launchers that dispatch the storage-typed passes to the
// per-storage translation units (lbm_st_*.cu).
#include "lbm_internal.cuh"

namespace hmcsc {
namespace {

// Tiled node index of linear node n = x + nx (y + ny z).
__device__ __forceinline__ long long tiled_of_linear(const StepParams &p,
                                                     long long n) {
  const int x = (int)(n % p.nx);
  const long long yz = n / p.nx;
  return (yz * p.ntx + x / kTile) * kTile + x % kTile;
}

// n_s and the adhesion source a = G_ads,2 n_s in tiled order (per component
// when the workspace holds n_s,2).
__global__ void k_geometry(StepParams p, Workspace w,
                           const float *__restrict__ ns_lin,
                           const float *__restrict__ ns2_lin,
                           const float *__restrict__ gads2_lin) {
  const long long N = (long long)p.nx * p.ny * p.nz;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const long long tn = tiled_of_linear(p, n);
    if (!in_bounds(w.fault, tn, p.ntiles * kTile, kFaultGeometry)) continue;
    const float s = ns_lin[n];
    const float g = gads2_lin[n];
    w.ns[tn] = s;
    w.ads[tn] = g * s;
    if (w.ns2) {
      const float s2 = ns2_lin ? ns2_lin[n] : s;
      w.ns2[tn] = s2;
      w.ads2[tn] = g * s2;
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block partial sums of the observables (fixed grid, fixed order).
__global__ void __launch_bounds__(kRedThreads) k_reduce(StepParams p,
                                                        Workspace w) {
  double acc[kRedK];
#pragma unroll
  for (int k = 0; k < kRedK; ++k) acc[k] = 0.0;
  const long long NT = p.ntiles * kTile;
  const int *L = p.res.layers;
  for (long long tn = blockIdx.x * (long long)kRedThreads + threadIdx.x; tn < NT;
       tn += (long long)kRedBlocks * kRedThreads) {
    const long long t = tn / kTile;
    const int x = (int)(t % p.ntx) * kTile + (int)(tn % kTile);
    if (x >= p.nx) continue;
    const long long yz = t / p.ntx;
    const int y = (int)(yz % p.ny);
    const int z = (int)(yz / p.ny);
    const float2 r = w.rho[in_bounds(w.fault, tn, p.ntiles * kTile, kFaultRhoLoad) ? tn : 0];
    acc[0] += r.x;
    acc[1] += r.y;
    if (!isfinite(r.x) || !isfinite(r.y)) acc[10] += 1.0;
    const bool in[kFaces] = {L[0] && x < L[0], L[1] && x >= p.nx - L[1],
                             L[2] && y < L[2], L[3] && y >= p.ny - L[3],
                             L[4] && z < L[4], L[5] && z >= p.nz - L[5]};
    bool any = false;
    const double pr =
        ((double)r.x + (double)r.y + (double)p.G * (double)r.x * (double)r.y) / 3.0;
#pragma unroll
    for (int k = 0; k < kFaces; ++k)
      if (in[k]) {
        any = true;
        acc[4 + k] += pr;
      }
    if (!any) {
      const double wgt_fluid = 1.0 - (double)w.ns[tn];
      acc[3] += wgt_fluid;
      if (r.x >= 0.5f) acc[2] += wgt_fluid;
    }
  }
  __shared__ double sm[kRedThreads / 32][kRedK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRedK; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sm[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kRedK) {
    double t = 0.0;
    for (int wi = 0; wi < kRedThreads / 32; ++wi) t += sm[wi][threadIdx.x];
    w.red[blockIdx.x * kRedK + threadIdx.x] = t;
  }
}

__global__ void k_reduce_final(Workspace w) {
  const int k = threadIdx.x;
  if (k >= kRedK) return;
  double t = 0.0;
  for (int b = 0; b < kRedBlocks; ++b) t += w.red[b * kRedK + k];
  w.red[kRedBlocks * kRedK + k] = t;
}

int flat_blocks(const StepParams &p) {
  long long N = (long long)p.nx * p.ny * p.nz;
  long long b = (N + 255) / 256;
  return (int)(b < 4864 ? (b < 1 ? 1 : b) : 4864);
}

}  // namespace

size_t workspace_bytes(long long nx, long long ny, long long nz, int storage,
                       bool per_component, Workspace *out, char *base) {
  const Tiling t = tiling(nx, ny, nz);
  const size_t nt = (size_t)t.ntiles * kTile;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  size_t o_f = take((size_t)storage_bytes(storage) * (size_t)t.ntiles * kTileFloats);
  size_t o_rho = take(sizeof(float2) * nt);
  size_t o_rho2 = take(storage_local(storage) ? sizeof(float2) * nt : 0);
  size_t o_ns = take(sizeof(float) * nt);
  size_t o_ads = take(sizeof(float) * nt);
  size_t o_stage = take(sizeof(float) * 6 * (size_t)t.nlin);
  size_t o_red = take(sizeof(double) * (kRedBlocks + 1) * kRedK);
  size_t o_ns2 = take(per_component ? sizeof(float) * nt : 0);
  size_t o_ads2 = take(per_component ? sizeof(float) * nt : 0);
  size_t o_fault = take(sizeof(unsigned));
  size_t o_wave = take(sizeof(unsigned) * (kWaveCtlWords + wave_flag_words(nx, ny, nz)));
  if (out) {
    out->f = (void *)(base + o_f);
    out->rho = (float2 *)(base + o_rho);
    out->rho_enc = storage_local(storage) ? (float2 *)(base + o_rho2) : nullptr;
    out->ns = (float *)(base + o_ns);
    out->ads = (float *)(base + o_ads);
    out->stage = (float *)(base + o_stage);
    out->red = (double *)(base + o_red);
    out->ns2 = per_component ? (float *)(base + o_ns2) : nullptr;
    out->ads2 = per_component ? (float *)(base + o_ads2) : nullptr;
    out->fault = (unsigned *)(base + o_fault);
    out->wave = (unsigned *)(base + o_wave);
    out->fault_host = nullptr;
  }
  return off;
}

cudaError_t launch_geometry(const StepParams &p, const Workspace &w,
                            const float *ns_lin, const float *ns2_lin,
                            const float *gads2_lin, cudaStream_t s) {
  k_geometry<<<flat_blocks(p), 256, 0, s>>>(p, w, ns_lin, ns2_lin, gads2_lin);
  return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(const StepParams &p, const Workspace &w,
                                    const float *rho_a, const float *rho_b,
                                    cudaStream_t s) {
  switch (p.storage) {
    case kF16: return launch_init_f16(p, w, rho_a, rho_b, s);
    case kBF16: return launch_init_bf16(p, w, rho_a, rho_b, s);
    case kF16L: return launch_init_f16l(p, w, rho_a, rho_b, s);
    case kBF16L: return launch_init_bf16l(p, w, rho_a, rho_b, s);
    default: return launch_init_f32(p, w, rho_a, rho_b, s);
  }
}

cudaError_t launch_density(const StepParams &p, const Workspace &w, int parity,
                           int cfg, cudaStream_t s) {
  switch (p.storage) {
    case kF16: return launch_density_f16(p, w, parity, cfg, s);
    case kBF16: return launch_density_bf16(p, w, parity, cfg, s);
    case kF16L: return launch_density_f16l(p, w, parity, cfg, s);
    case kBF16L: return launch_density_bf16l(p, w, parity, cfg, s);
    default: return launch_density_f32(p, w, parity, cfg, s);
  }
}

cudaError_t launch_collide_stream(const StepParams &p, const Workspace &w,
                                  int parity, int cfg, cudaStream_t s) {
  switch (p.storage) {
    case kF16: return launch_collide_f16(p, w, parity, cfg, s);
    case kBF16: return launch_collide_bf16(p, w, parity, cfg, s);
    case kF16L: return launch_collide_f16l(p, w, parity, cfg, s);
    case kBF16L: return launch_collide_bf16l(p, w, parity, cfg, s);
    default: return launch_collide_f32(p, w, parity, cfg, s);
  }
}

cudaError_t launch_fields(const StepParams &p, const Workspace &w, int parity,
                          cudaStream_t s) {
  switch (p.storage) {
    case kF16: return launch_fields_f16(p, w, parity, s);
    case kBF16: return launch_fields_bf16(p, w, parity, s);
    case kF16L: return launch_fields_f16l(p, w, parity, s);
    case kBF16L: return launch_fields_bf16l(p, w, parity, s);
    default: return launch_fields_f32(p, w, parity, s);
  }
}

cudaError_t launch_single_pass(const StepParams &p, const Workspace &w, int parity,
                               int nzc, cudaStream_t s) {
  switch (p.storage) {
    case kF16: return launch_single_pass_f16(p, w, parity, nzc, s);
    case kBF16: return launch_single_pass_bf16(p, w, parity, nzc, s);
    case kF16L: return launch_single_pass_f16l(p, w, parity, nzc, s);
    case kBF16L: return launch_single_pass_bf16l(p, w, parity, nzc, s);
    default: return launch_single_pass_f32(p, w, parity, nzc, s);
  }
}

cudaError_t launch_wave(const StepParams &p, const Workspace &w, int parity,
                        int cfg, int lag, unsigned spin_limit, long long hold,
                        cudaStream_t s) {
  switch (p.storage) {
    case kF16: return launch_wave_f16(p, w, parity, cfg, lag, spin_limit, hold, s);
    case kBF16: return launch_wave_bf16(p, w, parity, cfg, lag, spin_limit, hold, s);
    case kF16L: return launch_wave_f16l(p, w, parity, cfg, lag, spin_limit, hold, s);
    case kBF16L: return launch_wave_bf16l(p, w, parity, cfg, lag, spin_limit, hold, s);
    default: return launch_wave_f32(p, w, parity, cfg, lag, spin_limit, hold, s);
  }
}

cudaError_t launch_wave_batch(const WaveJob &job, int storage, cudaStream_t s) {
  switch (storage) {
    case kF16: return launch_wave_batch_f16(job, s);
    case kBF16: return launch_wave_batch_bf16(job, s);
    case kF16L: return launch_wave_batch_f16l(job, s);
    case kBF16L: return launch_wave_batch_bf16l(job, s);
    default: return launch_wave_batch_f32(job, s);
  }
}

cudaError_t launch_batch_collide_pipe(const BatchArgs &a, int storage, int even_cfg,
                                      int odd_cfg, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (even_cfg < kCollidePipeFirst || odd_cfg < kCollidePipeFirst) return cudaErrorInvalidValue;
  switch (storage) {
    case kF16: return launch_batch_collide_pipe_f16(a, even_cfg, odd_cfg, s);
    case kBF16: return launch_batch_collide_pipe_bf16(a, even_cfg, odd_cfg, s);
    case kF16L: return launch_batch_collide_pipe_f16l(a, even_cfg, odd_cfg, s);
    case kBF16L: return launch_batch_collide_pipe_bf16l(a, even_cfg, odd_cfg, s);
    default: return launch_batch_collide_pipe_f32(a, even_cfg, odd_cfg, s);
  }
}

cudaError_t launch_batch_density(const BatchArgs &a, int storage, cudaStream_t s) {
  if (a.n <= 0 || a.prefix[a.n] <= 0) return cudaSuccess;
  switch (storage) {
    case kF16: return launch_batch_density_f16(a, s);
    case kBF16: return launch_batch_density_bf16(a, s);
    case kF16L: return launch_batch_density_f16l(a, s);
    case kBF16L: return launch_batch_density_bf16l(a, s);
    default: return launch_batch_density_f32(a, s);
  }
}

cudaError_t launch_batch_collide(const BatchArgs &a, int storage, cudaStream_t s) {
  if (a.n <= 0 || a.prefix[a.n] <= 0) return cudaSuccess;
  switch (storage) {
    case kF16: return launch_batch_collide_f16(a, s);
    case kBF16: return launch_batch_collide_bf16(a, s);
    case kF16L: return launch_batch_collide_f16l(a, s);
    case kBF16L: return launch_batch_collide_bf16l(a, s);
    default: return launch_batch_collide_f32(a, s);
  }
}

cudaError_t launch_reduce(const StepParams &p, const Workspace &w,
                          cudaStream_t s) {
  k_reduce<<<kRedBlocks, kRedThreads, 0, s>>>(p, w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, 32, 0, s>>>(w);
  return cudaGetLastError();
}

}  // namespace hmcsc
