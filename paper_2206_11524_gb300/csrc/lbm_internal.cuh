// lbm_internal.cuh -- device-side lattice, workspace layout and kernel
// launchers of the HMCSC D3Q19 library (sm_103a).  Internal to the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace hmcsc {

constexpr int kQ = 19;
constexpr int kFaces = 6;

// Populations are stored in x-tiles of 32 nodes (one warp): tile
// t = xt + ntx * (y + ny * z), xt = x / 32.  Inside a tile, slot i holds the
// pair (f_i,1, f_i,2) of both components for each of the 32 nodes:
// f[t][i][x % 32][sigma].  Both components of a direction always move
// together (same source, same destination in either AA parity), so one
// 8-byte (float32) or 4-byte (16-bit) access carries both, a warp's access
// to one slot of its tile is one contiguous run of 256 or 128 bytes, and
// every slot of a tile sits at a fixed offset from the tile's base.
constexpr int kTile = 32;
constexpr int kTileFloats = 2 * kQ * kTile;  // population values per tile
constexpr int kTilePairs = kQ * kTile;       // (sigma = 1, 2) pairs per tile

// Population storage.  F32 stores f_i.  The 16-bit formats store an offset
// f_i - w_i rho_ref and decode to float32 for all arithmetic:
//   *_OFFSET: rho_ref = rho0_sigma, one constant per component;
//   *_LOCAL:  rho_ref = rho_sigma(y, t) for a population of node y at time
//             t + 1, i.e. the owner's own density one step earlier, so the
//             stored value is the deviation from that node's previous rest
//             equilibrium and keeps 16-bit precision relative to each
//             component's own local density.  A reader decodes all of its
//             populations with its own previous density; a writer encodes
//             with the destination's current density, which the force
//             stencil loads anyway.
// Half offsets are stored scaled by 2^14 (exact), which keeps offsets down
// to ~1e-8 out of the half subnormal range; bfloat16 needs no scale.
enum StorageKind { kF32 = 0, kF16 = 1, kBF16 = 2, kF16L = 3, kBF16L = 4 };
__host__ __device__ constexpr int storage_bytes(int st) { return st == kF32 ? 4 : 2; }
__host__ __device__ constexpr bool storage_local(int st) { return st == kF16L || st == kBF16L; }
// weight class of direction i: 0 rest, 1 axis, 2 diagonal
__host__ __device__ constexpr int wclass(int i) {
  return i == 0 ? 0 : ((i <= 3 || (i >= 10 && i <= 12)) ? 1 : 2);
}

// Half offsets are kept scaled by 2^14 (see above).
constexpr float kHalfScale = 16384.0f, kHalfUnscale = 1.0f / 16384.0f;

// The stored pair (sigma = 1, 2) of one direction at one node.  enc_s
// takes the reference already multiplied by kScale (exact: a power of two),
// so the half encode is one fused multiply-add per value: f * 2^14 - r 2^14
// rounds to the same float as (f - r) * 2^14 because scaling by a power of
// two commutes with rounding.
template <int ST> struct Codec2;
template <> struct Codec2<kF32> {
  using T2 = float2;
  static constexpr float kScale = 1.0f;
  static __device__ __forceinline__ float2 dec(T2 v, float2) { return v; }
  static __device__ __forceinline__ T2 enc_s(float f1, float f2, float2) {
    return make_float2(f1, f2);
  }
  static __device__ __forceinline__ T2 enc(float f1, float f2, float2) {
    return make_float2(f1, f2);
  }
};
template <> struct Codec2<kF16> {
  using T2 = __half2;
  static constexpr float kScale = kHalfScale;
  static __device__ __forceinline__ float2 dec(T2 v, float2 r) {
    const float2 h = __half22float2(v);
    return make_float2(fmaf(h.x, kHalfUnscale, r.x), fmaf(h.y, kHalfUnscale, r.y));
  }
  static __device__ __forceinline__ T2 enc_s(float f1, float f2, float2 rs) {
    return __floats2half2_rn(fmaf(f1, kHalfScale, -rs.x), fmaf(f2, kHalfScale, -rs.y));
  }
  static __device__ __forceinline__ T2 enc(float f1, float f2, float2 r) {
    return enc_s(f1, f2, make_float2(r.x * kHalfScale, r.y * kHalfScale));
  }
};
template <> struct Codec2<kBF16> {
  using T2 = __nv_bfloat162;
  static constexpr float kScale = 1.0f;
  static __device__ __forceinline__ float2 dec(T2 v, float2 r) {
    const float2 h = __bfloat1622float2(v);
    return make_float2(r.x + h.x, r.y + h.y);
  }
  static __device__ __forceinline__ T2 enc_s(float f1, float f2, float2 r) {
    return __floats2bfloat162_rn(f1 - r.x, f2 - r.y);
  }
  static __device__ __forceinline__ T2 enc(float f1, float f2, float2 r) {
    return enc_s(f1, f2, r);
  }
};
template <> struct Codec2<kF16L> : Codec2<kF16> {};
template <> struct Codec2<kBF16L> : Codec2<kBF16> {};

// D3Q19 velocity set in the order of Eq. A.8: direction i + 9 is the
// opposite of direction i (i = 1..9).
__host__ __device__ constexpr int cx(int i) {
  constexpr int t[kQ] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0,
                         1, 0, 0, 1, 1, 1, 1, 0, 0};
  return t[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int t[kQ] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1,
                         0, 1, 0, 1, -1, 0, 0, 1, 1};
  return t[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int t[kQ] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1,
                         0, 0, 1, 0, 0, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
// Lattice weights w_i: 1/3 rest, 1/18 axis, 1/36 diagonal (Appendix A.3).
__host__ __device__ constexpr float wgt(int i) {
  return i == 0 ? (1.0f / 3.0f)
                : ((cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) == 1 ? (1.0f / 18.0f)
                                                                       : (1.0f / 36.0f));
}

// Reservoir description handed to kernels: layers per face (0 = none), the
// prescribed densities and velocity (zero for a density reservoir; the
// velocity boundary cells of the Couette flow otherwise).  Faces
// -x,+x,-y,+y,-z,+z; higher index wins.
struct Reservoirs {
  int layers[kFaces];
  float rho[kFaces][2];
  float u[kFaces][3];
  int any;
  int moving;  // some face has a nonzero velocity
};

// Float products and sums rounded one by one (no fused multiply-add on the
// device; the host side is compiled without contraction), so that device
// and host evaluate res_feq identically.
__host__ __device__ inline float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ inline float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}

// f^eq_i(rho, u) of Eq. A.3 (c_s^2 = 1/3) for a node held at a prescribed
// state, with every operation rounded on its own.
__host__ __device__ inline float res_feq(int i, float rho, float ux, float uy,
                                         float uz) {
  const float cu = add_rn(add_rn(cx(i) * ux, cy(i) * uy), cz(i) * uz);
  const float uu = add_rn(add_rn(mul_rn(ux, ux), mul_rn(uy, uy)), mul_rn(uz, uz));
  float poly = add_rn(1.0f, mul_rn(3.0f, cu));
  poly = add_rn(poly, mul_rn(4.5f, mul_rn(cu, cu)));
  poly = add_rn(poly, -mul_rn(1.5f, uu));
  return mul_rn(mul_rn(wgt(i), rho), poly);
}

// Per-launch constants.  `res` lists the reservoirs whose reset ended the
// previous step; kernels read a node inside one of them as its equilibrium.
struct StepParams {
  int nx, ny, nz;
  int ntx;           // tiles along x: ceil(nx / 32)
  long long ntiles;  // ntx * ny * nz
  long long nlin;    // plane stride of the linear staging buffer
  float omega[2];    // 1 / tau_sigma
  float tau[2];
  float G;
  float F[3];
  float ref[2][3];   // *_OFFSET storages: w_class * rho0_sigma (float product)
  int storage;       // StorageKind
  Reservoirs res;
};

// Device workspace carved out of the caller's buffer.  Tiled arrays are
// indexed by tiled node index t * 32 + x % 32 (padding lanes x >= nx unused).
struct Workspace {
  void *f;           // [ntiles][38][32] populations (storage type), AA layout at parity t & 1
  float2 *rho;       // [ntiles * 32] (rho_1, rho_2) of the current time step
  float2 *rho_enc;   // [ntiles * 32] *_LOCAL storages: each node's density of
                     // the previous step, which its stored populations are
                     // offset from
  float *ns;         // [ntiles * 32] bounce-back fraction n_s (n_s,1 when the
                     // fractions are per component)
  float *ads;        // [ntiles * 32] a = G_ads,2 * n_s (adhesion stencil source;
                     // G_ads,2 n_s,1 when per component)
  float *ns2;        // [ntiles * 32] n_s,2, or nullptr: one fraction for both
  float *ads2;       // [ntiles * 32] G_ads,2 * n_s,2, or nullptr
  float *stage;      // [6][nlin] linear (x fastest) staging for host transfers
  double *red;       // [kRedBlocks][kRedK] partial sums + [kRedK] result
  unsigned *fault;   // bits of the accesses that were out of range in
                     // bounds-checked builds, and of wavefront waits that
                     // ran out in any build (FaultBits)
  unsigned *wave;    // wavefront step: kWaveCtlWords control words (ticket,
                     // blocks done, epoch, epoch of a launch whose wait ran
                     // out), then the tiles' flags
  unsigned *fault_host;  // host-mapped word that a wavefront wait which ran
                         // out also sets (read by lbm_step without waiting
                         // for the stream), or nullptr
};

// Bounds-checked builds (compiled with -DHMCSC_CHECKED) test the index of
// every population, density, geometry, staging and shared-ring access before
// making it; an index out of range sets a bit in the workspace's fault word
// and the access is skipped (a load reads element 0 instead).  Default
// builds compile the tests away.
enum FaultBits : unsigned {
  kFaultPopLoad = 1u, kFaultPopStore = 2u, kFaultRhoLoad = 4u,
  kFaultRhoStore = 8u, kFaultGeometry = 16u, kFaultShared = 32u,
  kFaultStage = 64u, kFaultWait = 128u, kFaultFlag = 256u
};
#ifdef HMCSC_CHECKED
constexpr bool kChecked = true;
__device__ __forceinline__ bool in_bounds(unsigned *fault, long long i, long long n,
                                          unsigned bit) {
  if (i >= 0 && i < n) return true;
  atomicOr(fault, bit);
  return false;
}
#else
constexpr bool kChecked = false;
__device__ __forceinline__ bool in_bounds(unsigned *, long long, long long, unsigned) {
  return true;
}
#endif

// Wavefront step: control words ahead of the flags (one per tile of 32 x by
// nodes of a plane; room for one per x-tile), and the default and smallest
// lag (planes the densities run ahead of the collisions).
constexpr int kWaveCtlWords = 64, kWaveLagDefault = 4, kWaveLagMin = 3;
constexpr int kWaveConfigs = 4;  // shapes 1 .. kWaveConfigs - 1 (0: two passes)
__host__ __device__ inline long long wave_flag_words(long long nx, long long ny,
                                                     long long nz) {
  return nz * ny * ((nx + 31) / 32);
}

constexpr int kRedBlocks = 304;  // 2 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kRedK = 11;        // mass[2], sat num/den, p_face[6], nonfinite

// Tiling of an nx x ny x nz lattice.
struct Tiling {
  long long ntx, ntiles, nlin;
};
__host__ __device__ inline Tiling tiling(long long nx, long long ny, long long nz) {
  Tiling t;
  t.ntx = (nx + kTile - 1) / kTile;
  t.ntiles = t.ntx * ny * nz;
  t.nlin = (nx * ny * nz + 63) / 64 * 64;
  return t;
}

// per_component: room for n_s,2 and its adhesion source (Eq. 1 with a
// bounce-back fraction per component).
size_t workspace_bytes(long long nx, long long ny, long long nz, int storage,
                       bool per_component, Workspace *out, char *base);

// Several lattices advanced by one launch per pass: block b of the grid
// belongs to item r with prefix[r] <= b < prefix[r + 1]; an item's blocks
// tile its lattice as 32 x 4 x 1 nodes.  Passed by value as a kernel
// parameter (about 16 KB for kBatchMax items).
constexpr int kBatchMax = 64;
constexpr int kBatchBY = 4;
struct BatchItem {
  StepParams p;
  Workspace w;
  int parity;  // AA parity of this lattice's current time step
  int gx, gy;  // blocks along x and y
};
struct BatchArgs {
  int n;
  int prefix[kBatchMax + 1];
  BatchItem item[kBatchMax];
};
static_assert(sizeof(BatchArgs) <= 32000, "kernel parameter limit");
cudaError_t launch_batch_density(const BatchArgs &a, int storage, cudaStream_t s);
cudaError_t launch_batch_collide(const BatchArgs &a, int storage, cudaStream_t s);
// The prefetching fused pass over a batch (k_batch_collide_pipe): one launch
// per AA parity present among the items, shapes even_cfg / odd_cfg (both >=
// kCollidePipeFirst); the items' gx, gy and the prefix table of `a` are
// not used (each launch lays out its own blocks).
cudaError_t launch_batch_collide_pipe(const BatchArgs &a, int storage, int even_cfg,
                                      int odd_cfg, cudaStream_t s);

// One batched wavefront step (k_wave_batch, one launch per AA parity
// present) over n lattices of one storage kind: lattice k's parameters,
// workspace and AA parity; wavefront shape cfg (1..kWaveConfigs - 1); lag >=
// kWaveLagMin.  spin_limit bounds the polls of one flag; hold names a flag
// of lattice 0 that the launch leaves unpublished (-1: none; tests of the
// failure path).
struct WaveJob {
  int n;
  const StepParams *sp[kBatchMax];
  const Workspace *ws[kBatchMax];
  int parity[kBatchMax];
  int cfg;
  int lag;
  unsigned spin_limit;
  long long hold;
};
constexpr unsigned kWaveSpinDefault = 1u << 22;
// Share of L2 that the planes in flight of one set of a batched wavefront
// launch may fill (lattices beyond it go to the next set).
constexpr double kWaveSetL2Share = 0.5;

// Per-storage launchers (one translation unit per storage kind).
#define HMCSC_DECLARE_STORAGE_LAUNCHERS(SUF)                                   \
  cudaError_t launch_density_##SUF(const StepParams &, const Workspace &, int, \
                                   int, cudaStream_t);                         \
  cudaError_t launch_collide_##SUF(const StepParams &, const Workspace &, int, \
                                   int, cudaStream_t);                         \
  cudaError_t launch_fields_##SUF(const StepParams &, const Workspace &, int,  \
                                  cudaStream_t);                               \
  cudaError_t launch_init_##SUF(const StepParams &, const Workspace &,         \
                                const float *, const float *, cudaStream_t);   \
  cudaError_t launch_single_pass_##SUF(const StepParams &, const Workspace &,  \
                                       int, int, cudaStream_t);                \
  cudaError_t launch_wave_##SUF(const StepParams &, const Workspace &, int,     \
                                int, int, unsigned, long long, cudaStream_t);  \
  cudaError_t launch_wave_batch_##SUF(const WaveJob &, cudaStream_t);         \
  cudaError_t launch_batch_density_##SUF(const BatchArgs &, cudaStream_t);     \
  cudaError_t launch_batch_collide_##SUF(const BatchArgs &, cudaStream_t);     \
  cudaError_t launch_batch_collide_pipe_##SUF(const BatchArgs &, int, int, cudaStream_t);
HMCSC_DECLARE_STORAGE_LAUNCHERS(f32)
HMCSC_DECLARE_STORAGE_LAUNCHERS(f16)
HMCSC_DECLARE_STORAGE_LAUNCHERS(bf16)
HMCSC_DECLARE_STORAGE_LAUNCHERS(f16l)
HMCSC_DECLARE_STORAGE_LAUNCHERS(bf16l)

// Kernel launchers (return the launch error).
cudaError_t launch_init_equilibrium(const StepParams &p, const Workspace &w,
                                    const float *rho_a, const float *rho_b,
                                    cudaStream_t s);
// ns2_lin may be nullptr (n_s,2 = n_s,1); it is read only when the
// workspace holds per-component fractions.
cudaError_t launch_geometry(const StepParams &p, const Workspace &w,
                            const float *ns_lin, const float *ns2_lin,
                            const float *gads2_lin, cudaStream_t s);
// `cfg` selects the launch shape of the pass (0 = default; see
// density_shape / collide_shape in lbm_device.cuh).
// Fused-pass shapes kCollidePipeFirst and up prefetch the next plane's
// populations into shared memory (k_collide_pipe, pipe_cfg).
constexpr int kDensityConfigs = 3, kCollideConfigs = 10, kCollidePipeFirst = 5;
cudaError_t launch_density(const StepParams &p, const Workspace &w, int parity,
                           int cfg, cudaStream_t s);
cudaError_t launch_collide_stream(const StepParams &p, const Workspace &w,
                                  int parity, int cfg, cudaStream_t s);
cudaError_t launch_fields(const StepParams &p, const Workspace &w, int parity,
                          cudaStream_t s);
// One whole step in a single sweep over the populations (bulk boxes of
// kSpBY rows x nz / nzc planes, then their seams); needs nx <= kSinglePassMaxNx
// and 1 <= nzc <= nz.
// Leaves the step's densities in w.rho like launch_density.
constexpr int kSinglePassMaxNx = 256;
cudaError_t launch_single_pass(const StepParams &p, const Workspace &w, int parity,
                               int nzc, cudaStream_t s);
// One whole step in one persistent launch (k_wave): densities computed lag
// planes ahead of the collision, the second read of the populations served
// by L2.  cfg in 1 .. kWaveConfigs - 1 (wave_cfg), lag >= kWaveLagMin.
// Leaves the step's densities in w.rho like launch_density.
cudaError_t launch_wave(const StepParams &p, const Workspace &w, int parity,
                        int cfg, int lag, unsigned spin_limit, long long hold,
                        cudaStream_t s);
cudaError_t launch_wave_batch(const WaveJob &job, int storage, cudaStream_t s);
cudaError_t launch_reduce(const StepParams &p, const Workspace &w,
                          cudaStream_t s);

}  // namespace hmcsc
