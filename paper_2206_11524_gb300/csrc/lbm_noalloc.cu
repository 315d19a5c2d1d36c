// lbm_noalloc.cu -- lbm_reduce_fields_noalloc: the observables of
// lbm_reduce computed from density fields in caller memory, using a fixed
// scratch array that lives in the library's own device image instead of a
// workspace.
//
// Who needs it: code that may not call cudaMalloc at the point where it wants
// the saturation and masses -- a host framework that hands out only its own
// fixed buffers, a real-time loop where an allocation would synchronise the
// device, or a plugin that never owns a workspace.  Such a caller passes its
// density and n_s fields and gets the numbers back; nothing is allocated.
//
// The scratch is the file-scope array g_noalloc_scratch below.  Every GPU
// that loads the library holds it (about 360 KB) until the process exits.
// All calls share it: two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it and may return wrong
// numbers.  Each call overwrites every slot it reads before reading it, so
// no clearing between calls is needed.
#include <mutex>

#include "lbm.h"
#include "lbm_internal.cuh"

namespace {
constexpr int kNoallocThreads = 256;
constexpr int kNodesPerBlock = 4096;  // 16 nodes per thread
constexpr int kNoallocMaxBlocks = LBM_NOALLOC_MAX_NODES / kNodesPerBlock;
constexpr int kK = hmcsc::kRedK;

static_assert(LBM_NOALLOC_MAX_NODES % kNodesPerBlock == 0, "max nodes");
}  // namespace

// Block partial sums [kNoallocMaxBlocks][kK], then the kK totals.
static __device__ __align__(256) double g_noalloc_scratch[(kNoallocMaxBlocks + 1) * kK];

namespace {

// Device address of g_noalloc_scratch per device, looked up once.  In host
// code the symbol's name is only a host-side stand-in, never a device
// address, so the address comes from cudaGetSymbolAddress.
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices];
std::mutex g_scratch_mu;

cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

struct FieldArgs {
  const float *rho1, *rho2, *ns;
  int nx, ny, nz;
  int layers[hmcsc::kFaces];
  double G;
  long long n;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Same per-node arithmetic as the workspace reduction: masses, non-finite
// count, S_1 numerator / denominator over nodes outside every reservoir, and
// the pressure sum of each reservoir face.  One block per 4096 nodes.
__global__ void __launch_bounds__(kNoallocThreads)
    k_reduce_fields(FieldArgs a, double *scratch) {
  double acc[kK];
#pragma unroll
  for (int k = 0; k < kK; ++k) acc[k] = 0.0;
  const long long first = (long long)blockIdx.x * kNodesPerBlock;
  long long last = first + kNodesPerBlock;
  if (last > a.n) last = a.n;
  const int *L = a.layers;
  for (long long n = first + threadIdx.x; n < last; n += kNoallocThreads) {
    const int x = (int)(n % a.nx);
    const int y = (int)((n / a.nx) % a.ny);
    const int z = (int)(n / ((long long)a.nx * a.ny));
    const float r1 = a.rho1[n], r2 = a.rho2[n];
    acc[0] += r1;
    acc[1] += r2;
    if (!isfinite(r1) || !isfinite(r2)) acc[10] += 1.0;
    const bool in[hmcsc::kFaces] = {L[0] && x < L[0], L[1] && x >= a.nx - L[1],
                                    L[2] && y < L[2], L[3] && y >= a.ny - L[3],
                                    L[4] && z < L[4], L[5] && z >= a.nz - L[5]};
    bool any = false;
    const double pr = ((double)r1 + (double)r2 + a.G * (double)r1 * (double)r2) / 3.0;
#pragma unroll
    for (int k = 0; k < hmcsc::kFaces; ++k)
      if (in[k]) {
        any = true;
        acc[4 + k] += pr;
      }
    if (!any) {
      const double w = 1.0 - (double)a.ns[n];
      acc[3] += w;
      if (r1 >= 0.5f) acc[2] += w;
    }
  }
  __shared__ double sm[kNoallocThreads / 32][kK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kK; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sm[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kK) {
    double t = 0.0;
    for (int w = 0; w < kNoallocThreads / 32; ++w) t += sm[w][threadIdx.x];
    scratch[blockIdx.x * kK + threadIdx.x] = t;
  }
}

__global__ void k_reduce_fields_final(double *scratch, int blocks) {
  const int k = threadIdx.x;
  if (k >= kK) return;
  double t = 0.0;
  for (int b = 0; b < blocks; ++b) t += scratch[b * kK + k];
  scratch[kNoallocMaxBlocks * kK + k] = t;
}

}  // namespace

extern "C" LBM_API lbm_status lbm_reduce_fields_noalloc(
    const float *d_rho_a, const float *d_rho_b, const float *d_ns, int32_t nx,
    int32_t ny, int32_t nz, const int32_t *layers, double G, void *cuda_stream,
    lbm_observables *out) {
  if (!d_rho_a || !d_rho_b || !d_ns || !out) return LBM_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1 || !(G == G)) return LBM_EINVAL;
  const long long N = (long long)nx * ny * nz;
  if (N > LBM_NOALLOC_MAX_NODES) return LBM_ETOOLARGE;
  FieldArgs a;
  a.rho1 = d_rho_a;
  a.rho2 = d_rho_b;
  a.ns = d_ns;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  // the pressure uses G rounded to float, as a context holds it, so the
  // result is the one lbm_reduce gives for the same state
  a.G = (double)(float)G;
  a.n = N;
  const int ext[3] = {nx, ny, nz};
  for (int k = 0; k < hmcsc::kFaces; ++k) {
    a.layers[k] = layers ? layers[k] : 0;
    if (a.layers[k] < 0 || a.layers[k] > ext[k / 2]) return LBM_EINVAL;
  }
  double *scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return LBM_ECUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int blocks = (int)((N + kNodesPerBlock - 1) / kNodesPerBlock);
  k_reduce_fields<<<blocks, kNoallocThreads, 0, s>>>(a, scratch);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  k_reduce_fields_final<<<1, 32, 0, s>>>(scratch, blocks);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  double r[kK];
  if (cudaMemcpyAsync(r, scratch + (size_t)kNoallocMaxBlocks * kK, sizeof r,
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return LBM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ECUDA;
  out->mass[0] = r[0];
  out->mass[1] = r[1];
  out->sat1 = r[3] > 0.0 ? r[2] / r[3] : NAN;
  for (int k = 0; k < hmcsc::kFaces; ++k) {
    if (a.layers[k] == 0) {
      out->p_face[k] = NAN;
      continue;
    }
    const long long cnt = (long long)a.layers[k] * (N / ext[k / 2]);
    out->p_face[k] = r[4 + k] / (double)cnt;
  }
  out->nonfinite = (int64_t)r[10];
  return out->nonfinite > 0 ? LBM_ENAN : LBM_OK;
}
