// lbm_internal.cuh -- device-side lattice, workspace layout and kernel
// launchers of the HMCSC D3Q19 library (sm_103a).  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace hmcsc {

constexpr int kQ = 19;
constexpr int kFaces = 6;

// Populations are stored in x-tiles of 32 nodes (one warp): tile
// t = xt + ntx * (y + ny * z), xt = x / 32, and inside a tile the 38 slots
// (sigma, i) are consecutive runs of 32 floats: f[t][sigma * 19 + i][x % 32].
// A warp's access to one slot of its tile is one aligned 128-byte line, and
// every slot of a tile sits at a fixed offset from the tile's base.
constexpr int kTile = 32;
constexpr int kTileFloats = 2 * kQ * kTile;

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

// Reservoir description handed to kernels: layers per face (0 = none) and
// the prescribed densities.  Faces -x,+x,-y,+y,-z,+z; higher index wins.
struct Reservoirs {
  int layers[kFaces];
  float rho[kFaces][2];
  int any;
};

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
  Reservoirs res;
};

// Device workspace carved out of the caller's buffer.  Tiled arrays are
// indexed by tiled node index t * 32 + x % 32 (padding lanes x >= nx unused).
struct Workspace {
  float *f;          // [ntiles][38][32] populations, AA layout at parity t & 1
  float2 *rho;       // [ntiles * 32] (rho_1, rho_2) of the current time step
  float *ns;         // [ntiles * 32] bounce-back fraction n_s
  float *ads;        // [ntiles * 32] a = G_ads,2 * n_s (adhesion stencil source)
  float *stage;      // [6][nlin] linear (x fastest) staging for host transfers
  double *red;       // [kRedBlocks][kRedK] partial sums + [kRedK] result
};

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

size_t workspace_bytes(long long nx, long long ny, long long nz, Workspace *out,
                       char *base);

// Kernel launchers (return the launch error).
cudaError_t launch_init_equilibrium(const StepParams &p, const Workspace &w,
                                    const float *rho_a, const float *rho_b,
                                    cudaStream_t s);
cudaError_t launch_geometry(const StepParams &p, const Workspace &w,
                            const float *ns_lin, const float *gads2_lin,
                            cudaStream_t s);
cudaError_t launch_density(const StepParams &p, const Workspace &w, int parity,
                           cudaStream_t s);
cudaError_t launch_collide_stream(const StepParams &p, const Workspace &w,
                                  int parity, cudaStream_t s);
cudaError_t launch_fields(const StepParams &p, const Workspace &w, int parity,
                          cudaStream_t s);
cudaError_t launch_reduce(const StepParams &p, const Workspace &w,
                          cudaStream_t s);

}  // namespace hmcsc
