/*
 * lbm.h -- C ABI of the GB300 (sm_103a) homogenized multi-component
 * Shan-Chen lattice Boltzmann library (HMCSC, arXiv 2206.11524).
 *
 * One context advances one two-component D3Q19 lattice with the update of
 * Eq. 1 (gray BGK with partial bounce-back of fraction n_s), the Shan-Chen
 * fluid-fluid force of Eq. 3, the fluid-solid adhesion force of Eq. 4, the
 * body-force split of Eq. 5 and the equilibrium-velocity shift of Eq. 6.
 *
 * Conventions for every entry point:
 *   - Lattice size nx, ny, nz >= 1; node index n = x + nx*(y + ny*z), x
 *     fastest.  N = nx*ny*nz.  The lattice is periodic on every axis; walls
 *     are n_s = 1 cells (Appendix A) and open faces are density reservoirs
 *     (lbm_set_bc, Sec. 4).
 *   - Populations are numbered in the D3Q19 order of Eq. A.8 (direction
 *     i + 9 is the opposite of direction i for i = 1..9); component 0 is
 *     fluid 1, component 1 is fluid 2.
 *   - Host arrays (float*, double*) are caller-owned and only read or written
 *     during the call.  Device memory is never allocated by the library: the
 *     caller passes one device workspace of lbm_workspace_bytes() bytes,
 *     which the library carves up and never frees.  lbm_destroy frees only
 *     the host-side context.
 *   - Every call returns an lbm_status; nothing aborts or throws.  After an
 *     error, lbm_last_error(ctx) holds a one-line message.
 *   - Work is enqueued on the CUDA stream given to lbm_create.  Calls that
 *     return host data (read_fields, reduce, get_populations, save) wait for
 *     that stream.  A context must not be used from two threads at once.
 */
#ifndef HMCSC_LBM_H
#define HMCSC_LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* an argument is out of range or NULL             */
  LBM_ENOMEM = 2,    /* workspace smaller than lbm_workspace_bytes()    */
  LBM_ECUDA = 3,     /* a CUDA runtime call failed (message has detail) */
  LBM_ENAN = 4,      /* a density became non-finite                     */
  LBM_ETIMEOUT = 5,  /* lbm_sync: the stream did not finish in time     */
  LBM_ESTATE = 6,    /* call out of order (e.g. step before geometry)   */
  LBM_EINTERNAL = 7, /* a kernel reported an internal inconsistency    */
  LBM_ETOOLARGE = 8  /* lattice beyond LBM_NOALLOC_MAX_NODES            */
} lbm_status;

typedef enum {
  LBM_STORAGE_F32 = 0,         /* populations stored as float32             */
  LBM_STORAGE_F16_OFFSET = 1,  /* f_i - w_i rho0_sigma stored as IEEE half   */
  LBM_STORAGE_BF16_OFFSET = 2, /* f_i - w_i rho0_sigma stored as bfloat16    */
  LBM_STORAGE_F16_LOCAL = 3,   /* f_i - w_i rho_sigma(x - c_i, t - 1) as half:
                                  the offset from the rest equilibrium of the
                                  node that wrote the population, at the step
                                  it wrote it (two density buffers)          */
  LBM_STORAGE_BF16_LOCAL = 4   /* the same, stored as bfloat16               */
} lbm_storage;

/* Model parameters (names of Table 1). */
typedef struct {
  int32_t nx, ny, nz;
  int32_t storage;   /* lbm_storage                                         */
  double tau[2];     /* relaxation times tau_1, tau_2 > 1/2         (Eq. 1) */
  double G;          /* G_inter,12 = G_inter,21                     (Eq. 3) */
  double F_ext[3];   /* body force on the mixture, split by Eq. 5           */
  double rho0[2];    /* offset reference per component for the 16-bit
                        storages (populations are kept as f_i - w_i rho0);
                        ignored for LBM_STORAGE_F32.  All arithmetic is
                        float32 whatever the storage.                       */
  int32_t ns_per_component; /* 1: the workspace holds a bounce-back fraction
                        per component, n_s,1 and n_s,2 (Eq. 1; membranes and
                        porous obstacles, Secs. 3.5 and 4), set with
                        lbm_set_geometry_per_component; 0: one n_s for both */
} lbm_params;

/* Observables of the current state (Sec. 4, Eqs. 18-19, Eq. A.6). */
typedef struct {
  double mass[2];    /* sum over all nodes of rho_1 and rho_2               */
  double sat1;       /* S_1 of Eq. 19: nodes outside every reservoir, each
                        weighted by 1 - n_s,1, counted when rho_1 >= 0.5;
                        NaN when that weight sums to zero                   */
  double p_face[6];  /* mean pressure (Eq. A.6) over each reservoir face's
                        layers, faces -x,+x,-y,+y,-z,+z; NaN if no reservoir.
                        Eq. 18's Delta p = inlet mean - outlet mean.        */
  int64_t nonfinite; /* nodes whose rho_1 or rho_2 is NaN or infinite       */
} lbm_observables;

typedef struct lbm_ctx lbm_ctx;

/* Bytes of device workspace a context with these parameters needs
 * (populations 2 x 19 x N values of the storage type, densities, geometry,
 * output staging and reduction scratch).  Returns 0 if the parameters are
 * invalid. */
LBM_API size_t lbm_workspace_bytes(const lbm_params *params);

/* Create a context.  d_workspace: device pointer, 256-byte aligned, at least
 * lbm_workspace_bytes(params) bytes, owned by the caller and kept alive until
 * lbm_destroy.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * The state starts unset: call lbm_set_geometry, then lbm_init_equilibrium or
 * lbm_set_populations, before stepping.  Errors: EINVAL (bad params, NULL
 * out), ENOMEM (workspace too small), ECUDA. */
LBM_API lbm_status lbm_create(const lbm_params *params, void *d_workspace,
                      size_t workspace_bytes, void *cuda_stream,
                      lbm_ctx **out);

/* Free the host context (never the workspace).  NULL is a no-op. */
LBM_API void lbm_destroy(lbm_ctx *ctx);

/* Static geometry (Sec. 2, Sec. 4): ns[N] = bounce-back fraction n_s in
 * [0, 1] (Eq. 1), gads2[N] = G_ads,2 per node (Eq. 4; G_ads,1 = -G_ads,2,
 * Table 1; NULL = all zero).  Host arrays, copied to the device.
 * EINVAL if any n_s is outside [0, 1] or not finite. */
LBM_API lbm_status lbm_set_geometry(lbm_ctx *ctx, const float *ns, const float *gads2);

/* Static geometry with a bounce-back fraction per component (Eq. 1 with
 * n_s,sigma; the adhesion indicator of Eq. 4 is s = n_s,sigma and Eq. 7
 * weights each component by 1 - n_s,sigma): ns1[N], ns2[N] in [0, 1],
 * gads2[N] as for lbm_set_geometry.  ns2 = NULL means n_s,2 = n_s,1.  The
 * context must have been created with ns_per_component = 1 when ns2 is not
 * NULL (EINVAL otherwise); such a context also accepts lbm_set_geometry,
 * which sets both fractions to ns.  A membrane that only fluid 1 may cross is
 * n_s,1 = 0, n_s,2 = 1 (Sec. 4).  Host arrays, copied to the device. */
LBM_API lbm_status lbm_set_geometry_per_component(lbm_ctx *ctx, const float *ns1,
                                                  const float *ns2,
                                                  const float *gads2);

/* Start from rest: f_i,sigma = f^eq_i(rho_sigma, u = 0) (Eq. A.3), time 0.
 * rho_a, rho_b: host [N], each > 0 and finite (EINVAL otherwise). */
LBM_API lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const float *rho_a,
                                const float *rho_b);

/* Set every population: f[2][19][N] (host, natural layout: f[s][i][n] is
 * f_i,s at node n), time 0.  EINVAL if a component density is <= 0. */
LBM_API lbm_status lbm_set_populations(lbm_ctx *ctx, const float *f);

/* Copy every population of the current time step to the host, in the
 * natural layout of lbm_set_populations.  Waits for the stream. */
LBM_API lbm_status lbm_get_populations(lbm_ctx *ctx, float *f);

/* Density reservoir on one face (Sec. 4): after every step the `layers`
 * outermost layers of face `face` (0..5 = -x,+x,-y,+y,-z,+z) hold
 * f^eq(rho_a / rho_b, u = 0).  layers = 0 removes it.  Where two faces'
 * layers overlap, the higher face index wins.  May be called between steps
 * (an inlet density ramp): the new values reset the layers at the end of the
 * next step.  The initial state of the layers is whatever was set.  EINVAL
 * if the layers exceed the axis length or a density is not positive. */
LBM_API lbm_status lbm_set_bc(lbm_ctx *ctx, int face, int layers, double rho_a,
                      double rho_b);

/* Velocity boundary cells on one face (the Couette flow of Sec. 3.1): like
 * lbm_set_bc, but the layers hold f^eq(rho_a / rho_b, u) of Eq. A.3 with the
 * prescribed velocity u = (ux, uy, uz) for both components, evaluated in
 * float32 with each operation rounded separately.  u = 0 is a density
 * reservoir.  EINVAL as for lbm_set_bc, or if a velocity component is not
 * finite or |u_d| >= 0.5. */
LBM_API lbm_status lbm_set_bc_velocity(lbm_ctx *ctx, int face, int layers,
                                       double rho_a, double rho_b, double ux,
                                       double uy, double uz);

/* Advance n_steps time steps (Eq. 1 plus the reservoirs), asynchronously on
 * the context's stream.  Each step launches the density pass and the fused
 * force/collide/bounce-back/stream pass, or the single-pass sweep when
 * lbm_set_single_pass enabled it, or the wavefront launch when
 * lbm_set_wavefront enabled it.  n_steps = 0 is a no-op.  EINTERNAL (and
 * nothing enqueued) when a device fault was reported for the current state:
 * by a synchronising call (below), or by a wavefront launch that already
 * ran, through a host-mapped word the kernel sets (no stream wait). */
LBM_API lbm_status lbm_step(lbm_ctx *ctx, int n_steps);

/* Single-pass stepping for lbm_step (planes > 0; 0 = two passes, the
 * default): each step reads every population once.  The lattice is cut into
 * boxes of full x-rows, 8 rows by `planes` planes; one launch marches every
 * box along z, computing the densities of the next plane into shared memory
 * and colliding the current plane's inner rows with them; the last row and
 * plane of each box (its seams, whose populations no other box may see
 * updated) are then updated by a second launch.  Results are bit-identical
 * to the two-pass step.  Needs nx <= 256 (EINVAL otherwise).  lbm_density /
 * lbm_collide_stream and the batched entry points keep the two passes. */
LBM_API lbm_status lbm_set_single_pass(lbm_ctx *ctx, int planes);

/* Wavefront stepping for lbm_step (shape > 0; 0 = two passes, the default;
 * it takes precedence over lbm_set_single_pass): each step is one persistent
 * cooperative launch over work items, a tile of 32 x by nodes of one plane
 * each (shape 1: by = 4, 2: by = 2, 3: by = 8), taken in plane order from an
 * atomic ticket.  An item sums the populations of one plane's tile into the
 * density array and collides and streams the tile `lag` planes behind it
 * once the densities that collision reads are published (flags in the
 * workspace), so the second read of each plane's populations comes from L2
 * instead of DRAM.  lag = 0 takes the default (4); other values must be
 * >= 3 (EINVAL otherwise); shapes outside 0..3 are EINVAL.  Results are
 * bit-identical to the two-pass step.  Contexts on the wavefront step also
 * advance together in one launch per step in lbm_batch_step.  Every wait in
 * the launch is bounded: a wait that runs out (which a correct launch never
 * does) leaves that step's result undefined, sets bit 128 (LBM_FAULT_WAIT)
 * of the word lbm_fault_word reads, in every build, and makes the next
 * synchronising call and lbm_step return EINTERNAL.  lbm_density /
 * lbm_collide_stream keep the two passes. */
#define LBM_WAVE_SHAPES 4
#define LBM_FAULT_WAIT 128u
LBM_API lbm_status lbm_set_wavefront(lbm_ctx *ctx, int shape, int lag);

/* For tests of the failure path of the wavefront step: spin_limit = polls
 * of one flag before a wait gives up (0 = the default, 2^22, seconds of
 * waiting); withhold_flag = index plane * T + (y / by) * ceil(nx / 32) +
 * x / 32, T = ceil(ny / by) * ceil(nx / 32), of one tile's density flag that
 * the launch then never publishes, so the collisions that read those
 * densities wait until their limit runs out (-1 = none, the default).  In a
 * batch they apply when this context is the first one.  EINVAL if the index
 * is outside the flag words. */
LBM_API lbm_status lbm_set_wavefront_limits(lbm_ctx *ctx, uint32_t spin_limit,
                                            int64_t withhold_flag);
/* The wavefront shape (0: off) and lag in use, to *shape and *lag (either
 * may be NULL).  Errors: EINVAL (NULL ctx). */
LBM_API lbm_status lbm_get_wavefront(const lbm_ctx *ctx, int *shape, int *lag);

/* The two halves of one step, for callers that time or interleave them:
 * lbm_density (rho_sigma of Eq. A.4 at every node) followed by
 * lbm_collide_stream (Eqs. 3-6, A.3, 1 and the reservoirs) is exactly one
 * lbm_step(ctx, 1).  lbm_collide_stream without a preceding lbm_density at
 * the same time step is ESTATE. */
LBM_API lbm_status lbm_density(lbm_ctx *ctx);
LBM_API lbm_status lbm_collide_stream(lbm_ctx *ctx);

/* Time steps taken since the last init / set_populations / load. */
LBM_API int64_t lbm_time(const lbm_ctx *ctx);

/* Synchronising calls (lbm_read_fields, lbm_reduce, lbm_sync,
 * lbm_get_populations, lbm_save) read the fault word once the stream has
 * drained and return EINTERNAL when a bit is set: LBM_FAULT_WAIT (the state
 * is undefined) in any build, an out-of-range access in a bounds-checked
 * build.  Their outputs are filled all the same.  lbm_init_equilibrium,
 * lbm_set_populations and lbm_load replace the state and clear
 * LBM_FAULT_WAIT. */

/* Macroscopic fields of the current state, to host arrays (any may be NULL):
 * rho_a[N], rho_b[N] (Eq. A.4); u[3][N] = u_macro of Eq. 7 (x, y, z planes);
 * p[N] = c_s^2 (rho + G rho_1 rho_2) (Eq. A.6).  Waits for the stream. */
LBM_API lbm_status lbm_read_fields(lbm_ctx *ctx, float *rho_a, float *rho_b, float *u,
                           float *p);

/* Observables of the current state (FP64 accumulation, fixed summation
 * order, so repeated calls on the same state give identical bits).  Waits
 * for the stream.  Returns ENAN (after filling *out) if nonfinite > 0. */
LBM_API lbm_status lbm_reduce(lbm_ctx *ctx, lbm_observables *out);

/* Wait for the context's stream, polling; ETIMEOUT after timeout_s seconds
 * (the work stays queued; the context remains usable). */
LBM_API lbm_status lbm_sync(lbm_ctx *ctx, double timeout_s);

/* Checkpoint: lbm_checkpoint_bytes() bytes hold the lattice size, storage,
 * time step and every population in the device's own layout; lbm_load
 * restores them into a context created with the same lattice size and
 * storage (EINVAL otherwise, or when the header does not check).  Resuming
 * from a checkpoint reproduces the uninterrupted run bit for bit. */
LBM_API size_t lbm_checkpoint_bytes(const lbm_ctx *ctx);
LBM_API lbm_status lbm_save(lbm_ctx *ctx, void *host_buf, size_t bytes);
LBM_API lbm_status lbm_load(lbm_ctx *ctx, const void *host_buf, size_t bytes);

/* Message of the last error on this context ("" if none). */
LBM_API const char *lbm_last_error(const lbm_ctx *ctx);

/* Launch shapes of the density pass (0..LBM_DENSITY_CONFIGS-1) and of the
 * fused pass on even and odd steps (0..LBM_COLLIDE_CONFIGS-1): thread-block
 * shape and register budget; fused shape 4 stores with the streaming cache
 * policy; fused shapes 5-9 walk runs of planes per block and copy the next
 * plane's populations (shapes 8-9: and the neighbour densities) into shared
 * memory while colliding the current one (shape 9: with streaming stores).
 * A new context starts with the shapes measured fastest for its storage on
 * a 256^3 lattice (float32 1/6/7, half and bfloat16 offsets 0/6/8, local
 * offsets 0/9/9).  Results do not depend on the choice; speed does (the
 * autotuner measures them per lattice size and storage).  EINVAL if out of
 * range. */
#define LBM_DENSITY_CONFIGS 3
#define LBM_COLLIDE_CONFIGS 10
LBM_API lbm_status lbm_set_launch_config(lbm_ctx *ctx, int density_cfg,
                                         int even_cfg, int odd_cfg);
/* The shapes in use (EINVAL if an argument is NULL). */
LBM_API lbm_status lbm_get_launch_config(const lbm_ctx *ctx, int *density_cfg,
                                         int *even_cfg, int *odd_cfg);

/* ---- Batched stepping of independent lattices ---------------------------
 * Several contexts (up to LBM_BATCH_MAX, same storage kind, geometry and
 * state set) advance together, whatever their sizes and AA parities: when
 * every context uses the wavefront step (lbm_set_wavefront), each step is
 * one persistent wavefront launch over the tiles of all the lattices at
 * each AA parity present (in the first context's shape and lag; the
 * lattices are numbered group by group in sets whose planes in flight fit
 * half of L2); otherwise one density launch covers every lattice, and the
 * fused pass is one launch per AA parity present in the first context's
 * fused-pass shapes (the prefetching shapes 5..9 of lbm_set_launch_config;
 * with another shape, one plain launch over every lattice).  Each lattice
 * computes exactly what lbm_step computes for it alone.  Work goes
 * on `cuda_stream`; the contexts' own streams are not used, so the caller
 * orders the batch after earlier work on them.  EINVAL: bad count, NULL or
 * repeated context, mixed storage; ESTATE: a context without geometry or
 * state; EINTERNAL: a context whose state a wavefront wait left undefined. */
#define LBM_BATCH_MAX 64
LBM_API lbm_status lbm_batch_step(lbm_ctx *const *ctxs, int n, int n_steps,
                                  void *cuda_stream);

/* A CUDA graph of n_steps (even, >= 2) batched steps of the given contexts,
 * captured on cuda_stream (not the legacy default stream).  Launching it
 * runs those steps and advances every context's host state; it is valid as
 * long as each context still has the time parity, density buffers and
 * reservoirs it had at capture (after an even number of steps they return),
 * else the launch returns ESTATE and nothing runs.  Reservoir changes must
 * have taken effect (one step after lbm_set_bc) before capture.  The graph
 * refers to the contexts: destroy it before them. */
typedef struct lbm_graph lbm_graph;
LBM_API lbm_status lbm_batch_graph_create(lbm_ctx *const *ctxs, int n,
                                          int n_steps, void *cuda_stream,
                                          lbm_graph **out);
LBM_API lbm_status lbm_batch_graph_launch(lbm_graph *graph, void *cuda_stream);
LBM_API void lbm_batch_graph_destroy(lbm_graph *graph);

/* ---- Bounds-checked builds -------------------------------------------------
 * The library can be compiled with -DHMCSC_CHECKED (build.build(checked=True)):
 * every population, density, geometry, staging and shared-memory index is
 * then tested before the access, and an index out of range sets a bit in a
 * fault word kept in the workspace (1 population load, 2 population store,
 * 4 density load, 8 density store, 16 geometry, 32 shared ring, 64 staging,
 * 256 wavefront flag) instead of being used.  lbm_build_checked() returns 1
 * in such a build, 0 otherwise.  lbm_fault_word copies the word to *out
 * after waiting for the context's stream, and zeroes it when clear != 0; in
 * a default build only LBM_FAULT_WAIT (a wavefront wait that ran out) can
 * set it.  Errors: EINVAL (NULL), ECUDA. */
LBM_API int lbm_build_checked(void);
LBM_API lbm_status lbm_fault_word(lbm_ctx *ctx, uint32_t *out, int clear);

/* ---- Allocation-free observables -----------------------------------------
 * The paper has no counterpart to this entry point: it exists for callers
 * that cannot call cudaMalloc where they need the observables -- a host
 * framework that only lends out its own fixed buffers, a real-time loop in
 * which an allocation would stall the device, a plugin that never owns a
 * workspace.  It computes the same observables as lbm_reduce (the two
 * masses, the saturation, the reservoir mean pressures, the non-finite
 * count; see lbm_observables) from density fields the caller already holds
 * on the device, and allocates nothing: its scratch is a fixed array of
 * about 360 KB inside the library's device image, which every GPU that loads
 * the library keeps until the process exits.
 *
 *   d_rho_a, d_rho_b, d_ns  device arrays [N] (float32, x fastest), read only
 *   nx, ny, nz              lattice size, N = nx*ny*nz <= LBM_NOALLOC_MAX_NODES
 *                           (larger lattices return LBM_ETOOLARGE, nothing run)
 *   layers[6]               reservoir layers per face (-x,+x,-y,+y,-z,+z) as
 *                           given to lbm_set_bc; NULL = no reservoirs
 *   G                       the context's G, for the pressure; rounded to
 *                           float as a context holds it
 *   cuda_stream             stream to run on (NULL = legacy default stream)
 *   out                     host result; waits for the stream
 *
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one scratch array and it
 * keeps the last call's contents: calls whose work overlaps on the GPU
 * (other streams, other host threads) race and may return wrong numbers.
 * Returns EINVAL for NULL pointers or bad sizes, ECUDA on a CUDA error, ENAN
 * (after filling *out) when a density is non-finite. */
#define LBM_NOALLOC_MAX_NODES 16777216
LBM_API lbm_status lbm_reduce_fields_noalloc(const float *d_rho_a,
                                             const float *d_rho_b,
                                             const float *d_ns, int32_t nx,
                                             int32_t ny, int32_t nz,
                                             const int32_t *layers, double G,
                                             void *cuda_stream,
                                             lbm_observables *out);

#ifdef __cplusplus
}
#endif

#endif /* HMCSC_LBM_H */
