// lbm_api.cu -- host side of the C ABI declared in include/lbm.h.
//
// The context owns no device memory: it carves the caller's workspace into
// populations, densities, geometry, staging and reduction scratch, and
// enqueues kernels on the caller's stream.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lbm.h"
#include "lbm_internal.cuh"
#include "lbm_validate.h"

using hmcsc::kFaces;
using hmcsc::kQ;
using hmcsc::kRedBlocks;
using hmcsc::kRedK;

static_assert(LBM_BATCH_MAX == hmcsc::kBatchMax, "batch limit of the ABI");
static_assert(LBM_WAVE_SHAPES == hmcsc::kWaveConfigs, "wavefront shapes of the ABI");
static_assert(LBM_FAULT_WAIT == hmcsc::kFaultWait, "fault bit of the ABI");

struct lbm_ctx {
  lbm_params params;
  hmcsc::StepParams sp;   // sp.res: reservoirs applied at the end of the last step
  float2 *rho_buf[2];     // *_LOCAL storages: the two density buffers
  int enc;                // index of rho_buf holding the encoding densities
  hmcsc::Reservoirs res_current;  // reservoirs set by lbm_set_bc (next steps)
  hmcsc::Workspace ws;
  cudaStream_t stream;
  long long N;
  int64_t t;             // time steps since the state was set
  int64_t rho_at;        // time step of the densities in ws.rho (-1: none)
  bool have_geometry;
  bool have_state;
  uint64_t bc_version;    // bumped by every lbm_set_bc
  int launch_cfg[3];      // launch shapes: density, even fused, odd fused
  int single_pass_zc;     // > 0: lbm_step sweeps once, boxes of this many planes
  int wave_cfg;           // > 0: lbm_step is one wavefront launch of this shape
  int wave_lag;           // planes between a plane's density and its collision
  uint32_t wave_spin;     // polls of one flag before a wavefront wait gives up
  int64_t wave_hold;      // flag the warp-item launch leaves unpublished (-1)
  unsigned *fault_host;   // host-mapped word set by a wait that ran out, or NULL
  int fault_slot;         // its slot in the process-wide page (-1: none)
  bool fault_seen;        // a device fault was reported for the current state
  std::string err;
};

struct lbm_graph {
  std::vector<lbm_ctx *> ctxs;
  int steps;
  cudaGraphExec_t exec;
  std::vector<int> parity0;       // AA parity of each lattice at capture
  std::vector<int> enc0;          // encoding-density buffer index at capture
  std::vector<uint64_t> bc0;      // reservoir configuration at capture
};

namespace {

// Host-mapped fault words, one per context, from one pinned page allocated
// once per process (allocating and freeing pinned memory per context would
// synchronise the device every time a context is destroyed).
constexpr int kFaultSlots = 4096;
std::mutex g_fault_mu;
unsigned *g_fault_host = nullptr;     // host view of the page
unsigned *g_fault_dev = nullptr;      // its device view
bool g_fault_tried = false;
std::vector<int> g_fault_free;

// A slot's host and device pointers, or false when mapped host memory is
// unavailable or every slot is taken (the synchronising checks remain).
bool fault_slot_take(unsigned **host, unsigned **dev, int *slot) {
  std::lock_guard<std::mutex> lock(g_fault_mu);
  if (!g_fault_tried) {
    g_fault_tried = true;
    void *h = nullptr, *d = nullptr;
    if (cudaHostAlloc(&h, kFaultSlots * 16 * sizeof(unsigned), cudaHostAllocMapped) ==
        cudaSuccess) {
      if (cudaHostGetDevicePointer(&d, h, 0) == cudaSuccess) {
        memset(h, 0, kFaultSlots * 16 * sizeof(unsigned));
        g_fault_host = static_cast<unsigned *>(h);
        g_fault_dev = static_cast<unsigned *>(d);
        for (int k = kFaultSlots - 1; k >= 0; --k) g_fault_free.push_back(k);
      } else {
        cudaFreeHost(h);
      }
    }
    cudaGetLastError();  // a failed optional allocation is not an error
  }
  if (!g_fault_host || g_fault_free.empty()) return false;
  *slot = g_fault_free.back();
  g_fault_free.pop_back();
  // one word per 64-byte line, so contexts never share a line
  *host = g_fault_host + *slot * 16;
  *dev = g_fault_dev + *slot * 16;
  *(volatile unsigned *)*host = 0u;
  return true;
}

void fault_slot_give(int slot) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lock(g_fault_mu);
  g_fault_free.push_back(slot);
}

lbm_status fail(lbm_ctx *c, lbm_status s, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *what) {
  return fail(c, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool params_valid(const lbm_params *p, const char **why) {
  if (!p) { *why = "params is NULL"; return false; }
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) { *why = "nx, ny, nz must be >= 1"; return false; }
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > 2147483647LL) { *why = "nx*ny*nz must be < 2^31"; return false; }
  if ((p->ny + 3) / 4 > 65535 || (p->nz + 1) / 2 > 65535) { *why = "ny or nz too large"; return false; }
  const hmcsc::Tiling tl = hmcsc::tiling(p->nx, p->ny, p->nz);
  if (tl.ntiles * hmcsc::kTile > 2147483647LL ||
      tl.ntiles * (long long)hmcsc::kTileFloats > 4294967295LL) {
    *why = "lattice too large for 32-node x-tiles"; return false;
  }
  if (p->storage < LBM_STORAGE_F32 || p->storage > LBM_STORAGE_BF16_LOCAL) {
    *why = "unsupported storage"; return false;
  }
  if (!std::isfinite(p->rho0[0]) || !std::isfinite(p->rho0[1])) { *why = "rho0 must be finite"; return false; }
  for (int s = 0; s < 2; ++s)
    if (!(p->tau[s] > 0.5) || !std::isfinite(p->tau[s])) { *why = "tau must be finite and > 1/2"; return false; }
  if (!std::isfinite(p->G)) { *why = "G must be finite"; return false; }
  if (p->ns_per_component != 0 && p->ns_per_component != 1) {
    *why = "ns_per_component must be 0 or 1"; return false;
  }
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(p->F_ext[d])) { *why = "F_ext must be finite"; return false; }
  return true;
}

size_t lin_stride(const lbm_ctx *c) { return (size_t)c->sp.nlin; }
size_t pop_floats(const lbm_ctx *c) { return (size_t)c->sp.ntiles * hmcsc::kTileFloats; }
size_t pop_bytes(const lbm_ctx *c) {
  return pop_floats(c) * (size_t)hmcsc::storage_bytes(c->sp.storage);
}

// Host-side encode / decode of one population in the context's storage
// with the reference w_i rho_ref already formed (the same float operations
// the kernels use: subtract, round to nearest into half / bfloat16; decode
// by adding the reference back).
void encode(int storage, void *dst, size_t idx, float f, float ref) {
  if (storage == hmcsc::kF16 || storage == hmcsc::kF16L)
    static_cast<__half *>(dst)[idx] = __float2half_rn((f - ref) * hmcsc::kHalfScale);
  else if (storage == hmcsc::kBF16 || storage == hmcsc::kBF16L)
    static_cast<__nv_bfloat16 *>(dst)[idx] = __float2bfloat16_rn(f - ref);
  else
    static_cast<float *>(dst)[idx] = f;
}
float decode(int storage, const void *src, size_t idx, float ref) {
  if (storage == hmcsc::kF16 || storage == hmcsc::kF16L)
    return ref + __half2float(static_cast<const __half *>(src)[idx]) * hmcsc::kHalfUnscale;
  if (storage == hmcsc::kBF16 || storage == hmcsc::kBF16L)
    return ref + __bfloat162float(static_cast<const __nv_bfloat16 *>(src)[idx]);
  return static_cast<const float *>(src)[idx];
}

// Tiled node index of (x, y, z).
size_t tiled_node(const lbm_ctx *c, long long x, long long y, long long z) {
  const long long t = x / hmcsc::kTile + c->sp.ntx * (y + (long long)c->params.ny * z);
  return (size_t)t * hmcsc::kTile + (size_t)(x % hmcsc::kTile);
}

// Point the workspace's density views at the buffers of the current state.
void set_density_views(lbm_ctx *c) {
  if (!hmcsc::storage_local(c->sp.storage)) return;
  c->ws.rho_enc = c->rho_buf[c->enc];
  c->ws.rho = c->rho_buf[1 - c->enc];
}

// Reference of population i (component s) of node (x,y,z) for decoding or
// encoding it as stored: *_LOCAL uses the node's own previous density in
// rho_enc (host copy, tiled float2), *_OFFSET the constant table.
float stored_ref(const lbm_ctx *c, const float *rho_enc_host, int s, int i,
                 int x, int y, int z) {
  if (hmcsc::storage_local(c->sp.storage))
    return hmcsc::wgt(i) * rho_enc_host[2 * tiled_node(c, x, y, z) + s];
  return c->sp.ref[s][hmcsc::wclass(i)];
}

// Index (in stored values) of population (component s, direction i) = slot
// k = s * 19 + i of node (x, y, z): tile, direction, lane, component.
size_t pop_offset(const lbm_ctx *c, int k, long long x, long long y, long long z) {
  const long long t = x / hmcsc::kTile + c->sp.ntx * (y + (long long)c->params.ny * z);
  const int s = k / kQ, i = k % kQ;
  return (((size_t)t * kQ + (size_t)i) * hmcsc::kTile + (size_t)(x % hmcsc::kTile)) * 2 +
         (size_t)s;
}

int parity(const lbm_ctx *c) { return (int)(c->t & 1); }

// The fault word after the context's stream has drained: EINTERNAL (with a
// message) when a bit is set, which also makes lbm_step refuse to advance
// the state until it is replaced or the word cleared.
lbm_status check_fault(lbm_ctx *c) {
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, c->ws.fault, sizeof v, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fault word");
  if (c->fault_host && *(volatile unsigned *)c->fault_host) v |= hmcsc::kFaultWait;
  if (v == 0) return LBM_OK;
  c->fault_seen = true;
  if (v == hmcsc::kFaultWait)
    return fail(c, LBM_EINTERNAL,
                "a wavefront wait ran out (fault word 0x%x): the state is undefined; "
                "load a checkpoint or set a new state", v);
  return fail(c, LBM_EINTERNAL,
              "the bounds-checked build recorded an out-of-range access (fault word 0x%x)", v);
}

// A new state replaces one a wavefront wait may have left undefined: the
// wait bit goes (out-of-range bits of checked builds stay until cleared).
lbm_status clear_wait_fault(lbm_ctx *c) {
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, c->ws.fault, sizeof v, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && (v & hmcsc::kFaultWait)) {
    static const unsigned keep_mask = ~hmcsc::kFaultWait;
    v &= keep_mask;
    e = cudaMemcpyAsync(c->ws.fault, &v, sizeof v, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "fault word");
  if (c->fault_host) *(volatile unsigned *)c->fault_host = 0u;
  c->fault_seen = false;
  return LBM_OK;
}

// Reservoir face of node (x, y, z) for reservoir set r (higher face wins).
int reservoir_face(const hmcsc::Reservoirs &r, const lbm_params &p, int x,
                   int y, int z) {
  int face = -1;
  if (r.layers[0] && x < r.layers[0]) face = 0;
  if (r.layers[1] && x >= p.nx - r.layers[1]) face = 1;
  if (r.layers[2] && y < r.layers[2]) face = 2;
  if (r.layers[3] && y >= p.ny - r.layers[3]) face = 3;
  if (r.layers[4] && z < r.layers[4]) face = 4;
  if (r.layers[5] && z >= p.nz - r.layers[5]) face = 5;
  return face;
}

// Checkpoint header.
struct CkptHeader {
  char magic[8];
  int32_t version, storage;
  int32_t nx, ny, nz, pad;
  int64_t t, ntiles;
  hmcsc::Reservoirs applied;  // reservoirs whose reset ended step t
};
const char kMagic[8] = {'H', 'M', 'C', 'S', 'C', 'L', 'B', '4'};

lbm_status sync_stream(lbm_ctx *c, const char *what) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return LBM_OK;
}

// Upload n floats from host to a device staging plane (pageable copy).
lbm_status upload(lbm_ctx *c, float *dst, const float *src, size_t n) {
  cudaError_t e = cudaMemcpyAsync(dst, src, n * sizeof(float),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  return LBM_OK;
}

// Host bookkeeping after the fused pass of a step.
void finish_step(lbm_ctx *c) {
  // The reservoirs in force now reset their layers at the end of this step.
  c->sp.res = c->res_current;
  // *_LOCAL: the densities of this step are the encoding densities now.
  if (hmcsc::storage_local(c->sp.storage)) {
    c->enc = 1 - c->enc;
    set_density_views(c);
  }
  c->t += 1;
}

}  // namespace

extern "C" {

size_t lbm_workspace_bytes(const lbm_params *params) {
  const char *why = nullptr;
  if (!params_valid(params, &why)) return 0;
  return hmcsc::workspace_bytes(params->nx, params->ny, params->nz,
                                params->storage, params->ns_per_component != 0,
                                nullptr, nullptr);
}

lbm_status lbm_create(const lbm_params *params, void *d_workspace,
                      size_t workspace_bytes, void *cuda_stream,
                      lbm_ctx **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  const char *why = nullptr;
  if (!params_valid(params, &why)) return LBM_EINVAL;
  if (!d_workspace || ((uintptr_t)d_workspace & 255u)) return LBM_EINVAL;
  const size_t need = hmcsc::workspace_bytes(params->nx, params->ny, params->nz,
                                             params->storage,
                                             params->ns_per_component != 0,
                                             nullptr, nullptr);
  if (workspace_bytes < need) return LBM_ENOMEM;
  lbm_ctx *c = new lbm_ctx();
  c->params = *params;
  c->stream = (cudaStream_t)cuda_stream;
  c->N = (long long)params->nx * params->ny * params->nz;
  hmcsc::workspace_bytes(params->nx, params->ny, params->nz, params->storage,
                         params->ns_per_component != 0, &c->ws, (char *)d_workspace);
  hmcsc::StepParams &sp = c->sp;
  sp.nx = params->nx;
  sp.ny = params->ny;
  sp.nz = params->nz;
  const hmcsc::Tiling tl = hmcsc::tiling(params->nx, params->ny, params->nz);
  sp.ntx = (int)tl.ntx;
  sp.ntiles = tl.ntiles;
  sp.nlin = tl.nlin;
  for (int s = 0; s < 2; ++s) {
    sp.tau[s] = (float)params->tau[s];
    sp.omega[s] = (float)(1.0 / params->tau[s]);
  }
  sp.G = (float)params->G;
  sp.storage = params->storage;
  for (int s = 0; s < 2; ++s) {
    const float r0 = (float)params->rho0[s];
    sp.ref[s][0] = hmcsc::wgt(0) * r0;
    sp.ref[s][1] = hmcsc::wgt(1) * r0;
    sp.ref[s][2] = hmcsc::wgt(4) * r0;
  }
  for (int d = 0; d < 3; ++d) sp.F[d] = (float)params->F_ext[d];
  memset(&sp.res, 0, sizeof sp.res);
  memset(&c->res_current, 0, sizeof c->res_current);
  c->rho_buf[0] = c->ws.rho;
  c->rho_buf[1] = c->ws.rho_enc;
  c->enc = 1;
  set_density_views(c);
  c->t = 0;
  c->rho_at = -1;
  c->have_geometry = false;
  c->have_state = false;
  c->bc_version = 0;
  // start from the shapes measured fastest for the storage on the 256^3
  // electrode (the tuner refines them per size)
  const bool local = hmcsc::storage_local(params->storage);
  const bool f32 = params->storage == LBM_STORAGE_F32;
  c->launch_cfg[0] = f32 ? 1 : 0;
  c->launch_cfg[1] = local ? 9 : 6;
  c->launch_cfg[2] = local ? 9 : (f32 ? 7 : 8);
  c->single_pass_zc = 0;
  c->wave_cfg = 0;
  c->wave_lag = hmcsc::kWaveLagDefault;
  c->wave_spin = hmcsc::kWaveSpinDefault;
  c->wave_hold = -1;
  c->fault_seen = false;
  // A host word the kernels can set when a wavefront wait runs out, so that
  // lbm_step sees it without waiting for the stream (none where mapped host
  // memory is unavailable: the checks at the synchronising calls remain).
  c->fault_host = nullptr;
  c->fault_slot = -1;
  {
    unsigned *h = nullptr, *d = nullptr;
    int slot = -1;
    if (fault_slot_take(&h, &d, &slot)) {
      c->fault_host = h;
      c->ws.fault_host = d;
      c->fault_slot = slot;
    }
  }
  // Zero the whole workspace once so padding lanes hold defined values.
  cudaError_t e = cudaMemsetAsync(d_workspace, 0, need, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    delete c;
    return LBM_ECUDA;
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx) {
  if (!ctx) return;
  fault_slot_give(ctx->fault_slot);
  delete ctx;
}

lbm_status lbm_set_geometry_per_component(lbm_ctx *c, const float *ns1,
                                          const float *ns2, const float *gads2) {
  if (!c) return LBM_EINVAL;
  if (!ns1) return fail(c, LBM_EINVAL, "ns is NULL");
  if (ns2 && !c->ws.ns2)
    return fail(c, LBM_EINVAL,
                "per-component n_s needs a context created with ns_per_component = 1");
  const float *fields[2] = {ns1, ns2};
  for (int k = 0; k < 2; ++k)
    if (fields[k]) {
      const long long n = hmcsc::first_bad(fields[k], c->N, hmcsc::BadFraction{});
      if (n < c->N)
        return fail(c, LBM_EINVAL, "n_s,%d[%lld] = %g is outside [0, 1]", k + 1, n,
                    (double)fields[k][n]);
    }
  if (gads2) {
    const long long n = hmcsc::first_bad(gads2, c->N, hmcsc::BadFinite{});
    if (n < c->N) return fail(c, LBM_EINVAL, "gads2[%lld] is not finite", n);
  }
  const size_t L = lin_stride(c);
  lbm_status st = upload(c, c->ws.stage, ns1, (size_t)c->N);
  if (st) return st;
  if (gads2) {
    st = upload(c, c->ws.stage + L, gads2, (size_t)c->N);
    if (st) return st;
  } else {
    cudaError_t e = cudaMemsetAsync(c->ws.stage + L, 0, sizeof(float) * c->N, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  }
  if (ns2) {
    st = upload(c, c->ws.stage + 2 * L, ns2, (size_t)c->N);
    if (st) return st;
  }
  cudaError_t e = hmcsc::launch_geometry(c->sp, c->ws, c->ws.stage,
                                         ns2 ? c->ws.stage + 2 * L : nullptr,
                                         c->ws.stage + L, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "geometry kernel");
  st = sync_stream(c, "set_geometry");
  if (st) return st;
  c->have_geometry = true;
  c->rho_at = -1;
  return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx *c, const float *ns, const float *gads2) {
  return lbm_set_geometry_per_component(c, ns, nullptr, gads2);
}

lbm_status lbm_init_equilibrium(lbm_ctx *c, const float *rho_a,
                                const float *rho_b) {
  if (!c) return LBM_EINVAL;
  if (!rho_a || !rho_b) return fail(c, LBM_EINVAL, "density array is NULL");
  {
    const long long na = hmcsc::first_bad(rho_a, c->N, hmcsc::BadDensity{});
    const long long nb = hmcsc::first_bad(rho_b, c->N, hmcsc::BadDensity{});
    const long long n = na < nb ? na : nb;
    if (n < c->N)
      return fail(c, LBM_EINVAL, "densities at node %lld must be finite and > 0", n);
  }
  const size_t L = lin_stride(c);
  lbm_status st = upload(c, c->ws.stage, rho_a, (size_t)c->N);
  if (st) return st;
  st = upload(c, c->ws.stage + L, rho_b, (size_t)c->N);
  if (st) return st;
  cudaError_t e = hmcsc::launch_init_equilibrium(c->sp, c->ws, c->ws.stage,
                                                 c->ws.stage + L, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  st = sync_stream(c, "init_equilibrium");
  if (st) return st;
  st = clear_wait_fault(c);
  if (st) return st;
  memset(&c->sp.res, 0, sizeof c->sp.res);
  c->t = 0;
  c->rho_at = -1;
  c->have_state = true;
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx *c, const float *f) {
  if (!c) return LBM_EINVAL;
  if (!f) return fail(c, LBM_EINVAL, "f is NULL");
  const long long N = c->N;
  for (int s = 0; s < 2; ++s)
    for (long long n = 0; n < N; ++n) {
      float r = 0.0f;
      for (int i = 0; i < kQ; ++i) {
        const float v = f[((size_t)s * kQ + i) * N + n];
        if (!std::isfinite(v)) return fail(c, LBM_EINVAL, "population not finite");
        r += v;
      }
      if (!(r > 0.0f)) return fail(c, LBM_EINVAL, "component %d density <= 0 at node %lld", s, n);
    }
  std::vector<char> tiled(pop_bytes(c), 0);
  const int nx = c->params.nx, ny = c->params.ny, nz = c->params.nz;
  const bool local = hmcsc::storage_local(c->sp.storage);
  // *_LOCAL: the given state is offset from its own nodes' densities
  // (summed in direction order, as the kernels do).
  std::vector<float> rho_enc(local ? 2 * (size_t)c->sp.ntiles * hmcsc::kTile : 0, 0.0f);
  if (local)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
          for (int sg = 0; sg < 2; ++sg) {
            float r = 0.0f;
            for (int i = 0; i < kQ; ++i)
              r += f[((size_t)sg * kQ + i) * N + x + (size_t)nx * (y + (size_t)ny * z)];
            rho_enc[2 * tiled_node(c, x, y, z) + sg] = r;
          }
  for (int sg = 0; sg < 2; ++sg)
    for (int i = 0; i < kQ; ++i)
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x) {
            const int k = sg * kQ + i;
            encode(c->sp.storage, tiled.data(), pop_offset(c, k, x, y, z),
                   f[(size_t)k * N + x + (size_t)nx * (y + (size_t)ny * z)],
                   stored_ref(c, rho_enc.data(), sg, i, x, y, z));
          }
  cudaError_t e = cudaMemcpyAsync(c->ws.f, tiled.data(), tiled.size(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  if (local) {
    e = cudaMemcpyAsync(c->ws.rho_enc, rho_enc.data(), rho_enc.size() * sizeof(float),
                        cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  }
  lbm_status st = sync_stream(c, "set_populations");
  if (st) return st;
  st = clear_wait_fault(c);
  if (st) return st;
  memset(&c->sp.res, 0, sizeof c->sp.res);
  c->t = 0;
  c->rho_at = -1;
  c->have_state = true;
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx *c, float *f) {
  if (!c) return LBM_EINVAL;
  if (!f) return fail(c, LBM_EINVAL, "f is NULL");
  if (!c->have_state) return fail(c, LBM_ESTATE, "no state set");
  const long long N = c->N;
  std::vector<char> raw(pop_bytes(c));
  cudaError_t e = cudaMemcpyAsync(raw.data(), c->ws.f, raw.size(),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  const bool local = hmcsc::storage_local(c->sp.storage);
  std::vector<float> rho_enc(local ? 2 * (size_t)c->sp.ntiles * hmcsc::kTile : 0);
  if (local) {
    e = cudaMemcpyAsync(rho_enc.data(), c->ws.rho_enc, rho_enc.size() * sizeof(float),
                        cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  }
  lbm_status st = sync_stream(c, "get_populations");
  if (st) return st;
  const lbm_status fst = check_fault(c);
  const int nx = c->params.nx, ny = c->params.ny, nz = c->params.nz;
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < kQ; ++i)
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x) {
            const long long n = x + (long long)nx * (y + (long long)ny * z);
            float v;
            if (parity(c) == 0) {
              v = decode(c->sp.storage, raw.data(), pop_offset(c, s * kQ + i, x, y, z),
                         stored_ref(c, rho_enc.data(), s, i, x, y, z));
            } else {
              // population i of node n sits in slot opp(i) of node n - c_i
              const int xs = (x - hmcsc::cx(i) + nx) % nx;
              const int ys = (y - hmcsc::cy(i) + ny) % ny;
              const int zs = (z - hmcsc::cz(i) + nz) % nz;
              v = decode(c->sp.storage, raw.data(),
                         pop_offset(c, s * kQ + hmcsc::opp(i), xs, ys, zs),
                         stored_ref(c, rho_enc.data(), s, i, x, y, z));
            }
            if (c->sp.res.any) {
              // a node inside a reservoir holds its prescribed equilibrium
              // (see the kernels)
              const int face = reservoir_face(c->sp.res, c->params, x, y, z);
              if (face >= 0) {
                const hmcsc::Reservoirs &r = c->sp.res;
                v = r.moving ? hmcsc::res_feq(i, r.rho[face][s], r.u[face][0],
                                              r.u[face][1], r.u[face][2])
                             : hmcsc::wgt(i) * r.rho[face][s];
              }
            }
            f[((size_t)s * kQ + i) * N + n] = v;
          }
  return fst;
}

lbm_status lbm_set_bc_velocity(lbm_ctx *c, int face, int layers, double rho_a,
                               double rho_b, double ux, double uy, double uz) {
  if (!c) return LBM_EINVAL;
  if (!std::isfinite(ux) || !std::isfinite(uy) || !std::isfinite(uz) ||
      std::fabs(ux) >= 0.5 || std::fabs(uy) >= 0.5 || std::fabs(uz) >= 0.5)
    return fail(c, LBM_EINVAL, "boundary velocity must be finite and below 0.5");
  if (face < 0 || face >= kFaces) return fail(c, LBM_EINVAL, "face must be 0..5");
  const int len = face < 2 ? c->params.nx : (face < 4 ? c->params.ny : c->params.nz);
  if (layers < 0 || layers > len) return fail(c, LBM_EINVAL, "layers out of range");
  if (layers > 0 && (!(rho_a > 0) || !(rho_b > 0) || !std::isfinite(rho_a) ||
                     !std::isfinite(rho_b)))
    return fail(c, LBM_EINVAL, "reservoir densities must be finite and > 0");
  c->bc_version += 1;
  hmcsc::Reservoirs &r = c->res_current;
  r.layers[face] = layers;
  r.rho[face][0] = layers > 0 ? (float)rho_a : 0.0f;
  r.rho[face][1] = layers > 0 ? (float)rho_b : 0.0f;
  r.u[face][0] = layers > 0 ? (float)ux : 0.0f;
  r.u[face][1] = layers > 0 ? (float)uy : 0.0f;
  r.u[face][2] = layers > 0 ? (float)uz : 0.0f;
  int any = 0, moving = 0;
  for (int k = 0; k < kFaces; ++k) {
    any |= r.layers[k] > 0;
    moving |= r.layers[k] > 0 && (r.u[k][0] != 0.0f || r.u[k][1] != 0.0f || r.u[k][2] != 0.0f);
  }
  r.any = any;
  r.moving = moving;
  return LBM_OK;
}

lbm_status lbm_set_bc(lbm_ctx *c, int face, int layers, double rho_a,
                      double rho_b) {
  return lbm_set_bc_velocity(c, face, layers, rho_a, rho_b, 0.0, 0.0, 0.0);
}

lbm_status lbm_density(lbm_ctx *c) {
  if (!c) return LBM_EINVAL;
  if (!c->have_geometry || !c->have_state)
    return fail(c, LBM_ESTATE, "set geometry and state before stepping");
  cudaError_t e = hmcsc::launch_density(c->sp, c->ws, parity(c), c->launch_cfg[0], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "density kernel");
  c->rho_at = c->t;
  return LBM_OK;
}

lbm_status lbm_collide_stream(lbm_ctx *c) {
  if (!c) return LBM_EINVAL;
  if (c->rho_at != c->t)
    return fail(c, LBM_ESTATE, "lbm_density must precede lbm_collide_stream");
  cudaError_t e = hmcsc::launch_collide_stream(c->sp, c->ws, parity(c),
                                                c->launch_cfg[1 + parity(c)], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "collide/stream kernel");
  finish_step(c);
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *c, int n_steps) {
  if (!c) return LBM_EINVAL;
  if (n_steps < 0) return fail(c, LBM_EINVAL, "n_steps < 0");
  if (n_steps == 0) return LBM_OK;
  if (!c->have_geometry || !c->have_state)
    return fail(c, LBM_ESTATE, "set geometry and state before stepping");
  if (c->fault_seen || (c->fault_host && *(volatile unsigned *)c->fault_host)) {
    c->fault_seen = true;
    return fail(c, LBM_EINTERNAL,
                "a wavefront wait ran out in an earlier step: the state is undefined; "
                "load a checkpoint or set a new state");
  }
  for (int k = 0; k < n_steps; ++k) {
    if (c->wave_cfg > 0) {
      cudaError_t e = hmcsc::launch_wave(c->sp, c->ws, parity(c), c->wave_cfg, c->wave_lag,
                                         c->wave_spin, c->wave_hold, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "wavefront kernel");
      c->rho_at = c->t;
      finish_step(c);
      continue;
    }
    if (c->single_pass_zc > 0) {
      // runs of about single_pass_zc planes along z
      const int nz = c->params.nz;
      int nzc = (nz + c->single_pass_zc / 2) / c->single_pass_zc;
      nzc = nzc < 1 ? 1 : (nzc > nz ? nz : nzc);
      cudaError_t e = hmcsc::launch_single_pass(c->sp, c->ws, parity(c), nzc, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "single-pass kernels");
      c->rho_at = c->t;
      finish_step(c);
      continue;
    }
    lbm_status st = lbm_density(c);
    if (st) return st;
    st = lbm_collide_stream(c);
    if (st) return st;
  }
  return LBM_OK;
}

lbm_status lbm_set_single_pass(lbm_ctx *c, int planes) {
  if (!c) return LBM_EINVAL;
  if (planes < 0) return fail(c, LBM_EINVAL, "planes must be >= 0");
  if (planes > 0 && c->params.nx > hmcsc::kSinglePassMaxNx)
    return fail(c, LBM_EINVAL, "the single-pass step needs nx <= %d", hmcsc::kSinglePassMaxNx);
  c->single_pass_zc = planes;
  return LBM_OK;
}

lbm_status lbm_set_wavefront(lbm_ctx *c, int shape, int lag) {
  if (!c) return LBM_EINVAL;
  if (shape < 0 || shape >= hmcsc::kWaveConfigs)
    return fail(c, LBM_EINVAL, "wavefront shape must be in 0..%d", hmcsc::kWaveConfigs - 1);
  if (lag == 0) lag = hmcsc::kWaveLagDefault;
  if (lag < hmcsc::kWaveLagMin)
    return fail(c, LBM_EINVAL, "wavefront lag must be >= %d", hmcsc::kWaveLagMin);
  if (((long long)c->params.nz + lag) * c->sp.ntx * c->params.ny > 4294967295LL)
    return fail(c, LBM_EINVAL, "wavefront lag too large for this lattice");
  c->wave_cfg = shape;
  c->wave_lag = lag;
  return LBM_OK;
}

lbm_status lbm_set_wavefront_limits(lbm_ctx *c, uint32_t spin_limit, int64_t withhold_flag) {
  if (!c) return LBM_EINVAL;
  const long long nflags = (long long)c->params.nz * c->params.ny * c->sp.ntx;
  if (withhold_flag < -1 || withhold_flag >= nflags)
    return fail(c, LBM_EINVAL, "withheld flag out of range");
  c->wave_spin = spin_limit ? spin_limit : hmcsc::kWaveSpinDefault;
  c->wave_hold = withhold_flag;
  return LBM_OK;
}

lbm_status lbm_get_wavefront(const lbm_ctx *c, int *shape, int *lag) {
  if (!c) return LBM_EINVAL;
  if (shape) *shape = c->wave_cfg;
  if (lag) *lag = c->wave_lag;
  return LBM_OK;
}

int64_t lbm_time(const lbm_ctx *c) { return c ? c->t : -1; }

lbm_status lbm_read_fields(lbm_ctx *c, float *rho_a, float *rho_b, float *u,
                           float *p) {
  if (!c) return LBM_EINVAL;
  if (!c->have_geometry || !c->have_state)
    return fail(c, LBM_ESTATE, "no state set");
  cudaError_t e = hmcsc::launch_density(c->sp, c->ws, parity(c), c->launch_cfg[0], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "density kernel");
  c->rho_at = c->t;
  e = hmcsc::launch_fields(c->sp, c->ws, parity(c), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fields kernel");
  const size_t L = lin_stride(c);
  const size_t bytes = sizeof(float) * (size_t)c->N;
  float *dst[6] = {rho_a, rho_b, u, u ? u + c->N : nullptr,
                   u ? u + 2 * c->N : nullptr, p};
  for (int k = 0; k < 6; ++k) {
    if (!dst[k]) continue;
    e = cudaMemcpyAsync(dst[k], c->ws.stage + (size_t)k * L, bytes,
                        cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  }
  lbm_status st = sync_stream(c, "read_fields");
  if (st) return st;
  return check_fault(c);
}

lbm_status lbm_reduce(lbm_ctx *c, lbm_observables *out) {
  if (!c) return LBM_EINVAL;
  if (!out) return fail(c, LBM_EINVAL, "out is NULL");
  if (!c->have_geometry || !c->have_state)
    return fail(c, LBM_ESTATE, "no state set");
  cudaError_t e = hmcsc::launch_density(c->sp, c->ws, parity(c), c->launch_cfg[0], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "density kernel");
  c->rho_at = c->t;
  hmcsc::StepParams obs = c->sp;
  obs.res = c->res_current;
  e = hmcsc::launch_reduce(obs, c->ws, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce kernel");
  double r[kRedK];
  e = cudaMemcpyAsync(r, c->ws.red + (size_t)kRedBlocks * kRedK, sizeof r,
                      cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  lbm_status st = sync_stream(c, "reduce");
  if (st) return st;
  const lbm_status fst = check_fault(c);
  out->mass[0] = r[0];
  out->mass[1] = r[1];
  out->sat1 = r[3] > 0.0 ? r[2] / r[3] : NAN;
  const long long ext[3] = {c->params.nx, c->params.ny, c->params.nz};
  for (int k = 0; k < kFaces; ++k) {
    const int L = c->res_current.layers[k];
    if (L == 0) {
      out->p_face[k] = NAN;
      continue;
    }
    const int axis = k / 2;
    const long long cnt = (long long)L * (ext[0] * ext[1] * ext[2] / ext[axis]);
    out->p_face[k] = r[4 + k] / (double)cnt;
  }
  out->nonfinite = (int64_t)r[10];
  if (fst) return fst;
  if (out->nonfinite > 0)
    return fail(c, LBM_ENAN, "%lld nodes have non-finite densities",
                (long long)out->nonfinite);
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx *c, double timeout_s) {
  if (!c) return LBM_EINVAL;
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(c, e, "event create");
  e = cudaEventRecord(ev, c->stream);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_fail(c, e, "event record");
  }
  const auto t0 = std::chrono::steady_clock::now();
  lbm_status st = LBM_OK;
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      st = cuda_fail(c, e, "stream");
      break;
    }
    const double el = std::chrono::duration<double>(
                          std::chrono::steady_clock::now() - t0).count();
    if (el > timeout_s) {
      st = fail(c, LBM_ETIMEOUT, "stream not finished after %.3f s", timeout_s);
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  cudaEventDestroy(ev);
  if (st == LBM_OK) st = check_fault(c);
  return st;
}

// Bytes of the encoding densities a *_LOCAL checkpoint carries.
size_t enc_bytes(const lbm_ctx *c) {
  return hmcsc::storage_local(c->sp.storage)
             ? sizeof(float2) * (size_t)c->sp.ntiles * hmcsc::kTile
             : 0;
}

size_t lbm_checkpoint_bytes(const lbm_ctx *c) {
  if (!c) return 0;
  return sizeof(CkptHeader) + pop_bytes(c) + enc_bytes(c);
}

lbm_status lbm_save(lbm_ctx *c, void *host_buf, size_t bytes) {
  if (!c) return LBM_EINVAL;
  if (!host_buf || bytes < lbm_checkpoint_bytes(c))
    return fail(c, LBM_EINVAL, "checkpoint buffer too small");
  if (!c->have_state) return fail(c, LBM_ESTATE, "no state set");
  CkptHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kMagic, 8);
  h.version = 4;
  h.storage = c->params.storage;
  h.nx = c->params.nx;
  h.ny = c->params.ny;
  h.nz = c->params.nz;
  h.t = c->t;
  h.ntiles = c->sp.ntiles;
  h.applied = c->sp.res;
  memcpy(host_buf, &h, sizeof h);
  cudaError_t e = cudaMemcpyAsync((char *)host_buf + sizeof h, c->ws.f,
                                  pop_bytes(c),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  if (enc_bytes(c)) {
    e = cudaMemcpyAsync((char *)host_buf + sizeof h + pop_bytes(c), c->ws.rho_enc,
                        enc_bytes(c), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  }
  lbm_status st = sync_stream(c, "save");
  if (st) return st;
  return check_fault(c);
}

lbm_status lbm_load(lbm_ctx *c, const void *host_buf, size_t bytes) {
  if (!c) return LBM_EINVAL;
  if (!host_buf || bytes < sizeof(CkptHeader))
    return fail(c, LBM_EINVAL, "checkpoint buffer too small");
  CkptHeader h;
  memcpy(&h, host_buf, sizeof h);
  if (memcmp(h.magic, kMagic, 8) != 0 || h.version != 4)
    return fail(c, LBM_EINVAL, "not a checkpoint of this library");
  if (h.nx != c->params.nx || h.ny != c->params.ny || h.nz != c->params.nz ||
      h.storage != c->params.storage || h.ntiles != c->sp.ntiles || h.t < 0)
    return fail(c, LBM_EINVAL, "checkpoint lattice or storage differs");
  if (bytes < lbm_checkpoint_bytes(c))
    return fail(c, LBM_EINVAL, "checkpoint truncated");
  cudaError_t e = cudaMemcpyAsync(c->ws.f, (const char *)host_buf + sizeof h,
                                  pop_bytes(c),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  if (enc_bytes(c)) {
    e = cudaMemcpyAsync(c->ws.rho_enc, (const char *)host_buf + sizeof h + pop_bytes(c),
                        enc_bytes(c), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  }
  lbm_status st = sync_stream(c, "load");
  if (st) return st;
  st = clear_wait_fault(c);
  if (st) return st;
  c->t = h.t;
  c->sp.res = h.applied;
  c->rho_at = -1;
  c->have_state = true;
  return LBM_OK;
}

// ---- batched stepping ----

namespace {

// Do all lattices of a batch use the wavefront step?  Then the batch
// advances by one persistent launch per step and AA parity over every
// lattice, in the first context's wavefront shape and lag.
bool batch_is_wave(lbm_ctx *const *ctxs, int n) {
  for (int k = 0; k < n; ++k)
    if (ctxs[k]->wave_cfg <= 0) return false;
  return true;
}

lbm_status batch_check(lbm_ctx *const *ctxs, int n) {
  if (!ctxs || n < 1 || n > hmcsc::kBatchMax) return LBM_EINVAL;
  long long items = 0;
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return LBM_EINVAL;
    if (!ctxs[k]->have_geometry || !ctxs[k]->have_state) return LBM_ESTATE;
    if (ctxs[k]->sp.storage != ctxs[0]->sp.storage) return LBM_EINVAL;
    if ((ctxs[k]->ws.ns2 != nullptr) != (ctxs[0]->ws.ns2 != nullptr)) return LBM_EINVAL;
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return LBM_EINVAL;
    items += ((long long)ctxs[k]->params.nz + ctxs[0]->wave_lag) * ctxs[k]->sp.ntx *
             ctxs[k]->params.ny;
  }
  // the persistent batched launch numbers every row tile of every group
  if (batch_is_wave(ctxs, n) && items > 4294967295LL)
    return fail(ctxs[0], LBM_EINVAL, "batch too large for one wavefront launch");
  return LBM_OK;
}

// The state a lattice has after one more step (same bookkeeping as
// lbm_collide_stream).
void advance_one(lbm_ctx *c) {
  c->sp.res = c->res_current;
  if (hmcsc::storage_local(c->sp.storage)) {
    c->enc = 1 - c->enc;
    set_density_views(c);
  }
  c->rho_at = -1;
  c->t += 1;
}

// Enqueue n_steps steps of every lattice on stream s: per step one
// persistent wavefront launch over all lattices (when every context uses the
// row-per-warp wavefront step), else one batched density pass and one
// batched fused pass.
lbm_status batch_enqueue(lbm_ctx *const *ctxs, int n, int n_steps, cudaStream_t s) {
  if (batch_is_wave(ctxs, n)) {
    for (int k = 0; k < n; ++k)
      if (ctxs[k]->fault_seen || (ctxs[k]->fault_host && *(volatile unsigned *)ctxs[k]->fault_host)) {
        ctxs[k]->fault_seen = true;
        return fail(ctxs[k], LBM_EINTERNAL,
                    "a wavefront wait ran out in an earlier step: the state is undefined");
      }
    static thread_local hmcsc::WaveJob job;
    for (int step = 0; step < n_steps; ++step) {
      job.n = n;
      job.cfg = ctxs[0]->wave_cfg;
      job.lag = ctxs[0]->wave_lag;
      job.spin_limit = ctxs[0]->wave_spin;
      job.hold = ctxs[0]->wave_hold;
      for (int k = 0; k < n; ++k) {
        job.sp[k] = &ctxs[k]->sp;
        job.ws[k] = &ctxs[k]->ws;
        job.parity[k] = (int)(ctxs[k]->t & 1);
      }
      cudaError_t e = hmcsc::launch_wave_batch(job, ctxs[0]->sp.storage, s);
      if (e != cudaSuccess) {
        for (int k = 0; k < n; ++k) cuda_fail(ctxs[k], e, "batched wavefront kernel");
        return LBM_ECUDA;
      }
      for (int k = 0; k < n; ++k) advance_one(ctxs[k]);
    }
    return LBM_OK;
  }
  static thread_local hmcsc::BatchArgs a;  // ~16 KB: kept off the stack
  for (int step = 0; step < n_steps; ++step) {
    a.n = n;
    a.prefix[0] = 0;
    for (int k = 0; k < n; ++k) {
      lbm_ctx *c = ctxs[k];
      hmcsc::BatchItem &it = a.item[k];
      it.p = c->sp;
      it.w = c->ws;
      it.parity = (int)(c->t & 1);
      it.gx = c->sp.ntx;
      it.gy = (c->params.ny + hmcsc::kBatchBY - 1) / hmcsc::kBatchBY;
      a.prefix[k + 1] = a.prefix[k] + it.gx * it.gy * c->params.nz;
    }
    cudaError_t e = hmcsc::launch_batch_density(a, ctxs[0]->sp.storage, s);
    // the fused pass in the first context's shapes: prefetching shapes run
    // as one batched prefetching launch per AA parity present
    const int ecfg = ctxs[0]->launch_cfg[1], ocfg = ctxs[0]->launch_cfg[2];
    if (e == cudaSuccess) {
      if (ecfg >= hmcsc::kCollidePipeFirst && ocfg >= hmcsc::kCollidePipeFirst)
        e = hmcsc::launch_batch_collide_pipe(a, ctxs[0]->sp.storage, ecfg, ocfg, s);
      else
        e = hmcsc::launch_batch_collide(a, ctxs[0]->sp.storage, s);
    }
    if (e != cudaSuccess) {
      for (int k = 0; k < n; ++k) cuda_fail(ctxs[k], e, "batched kernel");
      return LBM_ECUDA;
    }
    for (int k = 0; k < n; ++k) advance_one(ctxs[k]);
  }
  return LBM_OK;
}

struct SavedState {
  int64_t t, rho_at;
  hmcsc::StepParams sp;
  hmcsc::Workspace ws;
  int enc;
};

}  // namespace

lbm_status lbm_batch_step(lbm_ctx *const *ctxs, int n, int n_steps,
                          void *cuda_stream) {
  lbm_status st = batch_check(ctxs, n);
  if (st) return st;
  if (n_steps < 0) return LBM_EINVAL;
  return batch_enqueue(ctxs, n, n_steps, (cudaStream_t)cuda_stream);
}

lbm_status lbm_batch_graph_create(lbm_ctx *const *ctxs, int n, int n_steps,
                                  void *cuda_stream, lbm_graph **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  lbm_status st = batch_check(ctxs, n);
  if (st) return st;
  if (n_steps < 2 || n_steps % 2 != 0 || !cuda_stream) return LBM_EINVAL;
  for (int k = 0; k < n; ++k)
    if (memcmp(&ctxs[k]->sp.res, &ctxs[k]->res_current, sizeof(hmcsc::Reservoirs)) != 0)
      return fail(ctxs[k], LBM_ESTATE, "a reservoir change is pending: step once first");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  std::vector<SavedState> saved(n);
  for (int k = 0; k < n; ++k)
    saved[k] = {ctxs[k]->t, ctxs[k]->rho_at, ctxs[k]->sp, ctxs[k]->ws, ctxs[k]->enc};
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(ctxs[0], e, "begin capture");
  st = batch_enqueue(ctxs, n, n_steps, s);
  cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  for (int k = 0; k < n; ++k) {   // nothing ran: restore the host state
    ctxs[k]->t = saved[k].t;
    ctxs[k]->rho_at = saved[k].rho_at;
    ctxs[k]->sp = saved[k].sp;
    ctxs[k]->ws = saved[k].ws;
    ctxs[k]->enc = saved[k].enc;
  }
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e2 != cudaSuccess) return cuda_fail(ctxs[0], e2, "end capture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(ctxs[0], e, "graph instantiate");
  lbm_graph *g = new lbm_graph();
  g->ctxs.assign(ctxs, ctxs + n);
  g->steps = n_steps;
  g->exec = exec;
  for (int k = 0; k < n; ++k) {
    g->parity0.push_back((int)(ctxs[k]->t & 1));
    g->enc0.push_back(ctxs[k]->enc);
    g->bc0.push_back(ctxs[k]->bc_version);
  }
  *out = g;
  return LBM_OK;
}

lbm_status lbm_batch_graph_launch(lbm_graph *g, void *cuda_stream) {
  if (!g) return LBM_EINVAL;
  const size_t n = g->ctxs.size();
  for (size_t k = 0; k < n; ++k) {
    lbm_ctx *c = g->ctxs[k];
    if ((int)(c->t & 1) != g->parity0[k] || c->enc != g->enc0[k] ||
        c->bc_version != g->bc0[k] ||
        memcmp(&c->sp.res, &c->res_current, sizeof(hmcsc::Reservoirs)) != 0)
      return fail(c, LBM_ESTATE, "lattice changed since the graph was captured");
  }
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(g->ctxs[0], e, "graph launch");
  for (size_t k = 0; k < n; ++k)
    for (int s = 0; s < g->steps; ++s) advance_one(g->ctxs[k]);
  return LBM_OK;
}

void lbm_batch_graph_destroy(lbm_graph *g) {
  if (!g) return;
  cudaGraphExecDestroy(g->exec);
  delete g;
}

lbm_status lbm_set_launch_config(lbm_ctx *c, int density_cfg, int even_cfg,
                                 int odd_cfg) {
  if (!c) return LBM_EINVAL;
  if (density_cfg < 0 || density_cfg >= hmcsc::kDensityConfigs || even_cfg < 0 ||
      even_cfg >= hmcsc::kCollideConfigs || odd_cfg < 0 || odd_cfg >= hmcsc::kCollideConfigs)
    return fail(c, LBM_EINVAL, "launch configuration out of range");
  c->launch_cfg[0] = density_cfg;
  c->launch_cfg[1] = even_cfg;
  c->launch_cfg[2] = odd_cfg;
  return LBM_OK;
}

lbm_status lbm_get_launch_config(const lbm_ctx *c, int *density_cfg, int *even_cfg,
                                 int *odd_cfg) {
  if (!c || !density_cfg || !even_cfg || !odd_cfg) return LBM_EINVAL;
  *density_cfg = c->launch_cfg[0];
  *even_cfg = c->launch_cfg[1];
  *odd_cfg = c->launch_cfg[2];
  return LBM_OK;
}

int lbm_build_checked(void) { return hmcsc::kChecked ? 1 : 0; }

lbm_status lbm_fault_word(lbm_ctx *c, uint32_t *out, int clear) {
  if (!c) return LBM_EINVAL;
  if (!out) return fail(c, LBM_EINVAL, "out is NULL");
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, c->ws.fault, sizeof v, cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess && clear) e = cudaMemsetAsync(c->ws.fault, 0, sizeof v, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fault word");
  lbm_status st = sync_stream(c, "fault word");
  if (st) return st;
  if (c->fault_host && *(volatile unsigned *)c->fault_host) v |= hmcsc::kFaultWait;
  if (clear) {
    if (c->fault_host) *(volatile unsigned *)c->fault_host = 0u;
    c->fault_seen = false;
  }
  *out = v;
  return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c) {
  return c ? c->err.c_str() : "context is NULL";
}

}  // extern "C"
