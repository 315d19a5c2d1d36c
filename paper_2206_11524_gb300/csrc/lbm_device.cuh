// lbm_device.cuh -- device code of the HMCSC D3Q19 kernels, shared by the
// per-storage translation units (lbm_st_*.cu) that instantiate it.
//
// One time step is two launches:
//   k_density        rho_sigma(x) = sum_i f_i,sigma(x)                (Eq. A.4)
//   k_collide_stream moments, Shan-Chen forces (Eqs. 3-5), equilibrium
//                    velocity (Eq. 6), equilibrium (Eq. A.3), gray collision
//                    with partial bounce-back (Eq. 1) and in-place streaming
//   (or k_collide_pipe, the same arithmetic with the next plane's
//   populations copied into shared memory ahead of use)
// plus, as options, the single-pass sweep (k_sp_bulk + k_sp_seams) and the
// batched kernels that advance many lattices per launch.
//
// Density reservoirs (Sec. 4) reset their layers to the equilibrium at rest
// after every step, velocity boundary cells (Sec. 3.1) to the equilibrium at
// their velocity.  No kernel writes that reset: every reader of a node's
// populations (both passes, the fields pass, the host read-back) takes the
// prescribed equilibrium for a node inside such a layer, which is the state
// the reset defines, and what neighbours streamed into its slots is never
// read.
// StepParams::res holds the reservoirs that were in effect at the end of the
// previous step.
//
// Populations live in 32-node x-tiles (see lbm_internal.cuh) and stream in
// place with the AA pattern:
//   even t: node n reads slot i at n, writes its post-collision f_i to slot
//           opp(i) at n (population i of node n + c_i at t + 1);
//   odd t:  node n reads population i from slot opp(i) at n - c_i, writes
//           its post-collision f_i to slot i at n + c_i.
// Every (slot, node) a thread writes is one it read itself, so the update is
// race-free in place, and after an odd step the layout is natural again.
// One warp is one tile, and both components of a direction travel as one
// pair: on even steps all 19 loads and 19 stores of a thread are one pointer
// plus a constant; on odd steps there is one pointer per neighbour offset,
// shared by the load and the store at that offset.
#pragma once
#include "lbm_internal.cuh"

namespace hmcsc {
namespace {


// Periodic neighbourhood of one node in tile coordinates.
struct Geo {
  int tx[3], ln[3];  // tile-x index and lane of x-1, x, x+1
  int yw[3], zw[3];  // y-1..y+1, z-1..z+1 (wrapped)
  int tr[3][3];      // first tile of row (y', z'): ntx * (y' + ny * z')
  __device__ __forceinline__ int tile(int dx, int dy, int dz) const {
    return tr[dy + 1][dz + 1] + tx[dx + 1];
  }
  // tiled node index of x + (dx, dy, dz)
  __device__ __forceinline__ int node(int dx, int dy, int dz) const {
    return tile(dx, dy, dz) * kTile + ln[dx + 1];
  }
  // pair offset of slot 0 of node x + (dx, dy, dz) in the population array
  // (fits 32 bits: the host requires ntiles * 1216 < 2^32)
  __device__ __forceinline__ unsigned pop_off(int dx, int dy, int dz) const {
    return (unsigned)tile(dx, dy, dz) * (unsigned)kTilePairs + (unsigned)ln[dx + 1];
  }
};

__device__ __forceinline__ Geo make_geo(const StepParams &p, int x, int y,
                                        int z) {
  Geo g;
  const int xm = x == 0 ? p.nx - 1 : x - 1;
  const int xp = x == p.nx - 1 ? 0 : x + 1;
  g.tx[0] = xm / kTile; g.ln[0] = xm % kTile;
  g.tx[1] = x / kTile;  g.ln[1] = x % kTile;
  g.tx[2] = xp / kTile; g.ln[2] = xp % kTile;
  g.yw[0] = y == 0 ? p.ny - 1 : y - 1;
  g.yw[1] = y;
  g.yw[2] = y == p.ny - 1 ? 0 : y + 1;
  g.zw[0] = z == 0 ? p.nz - 1 : z - 1;
  g.zw[1] = z;
  g.zw[2] = z == p.nz - 1 ? 0 : z + 1;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) g.tr[a][b] = p.ntx * (g.yw[a] + p.ny * g.zw[b]);
  return g;
}

// Decode references of population i of node x (both components): w_i times
// the node's own previous density (*_LOCAL) or the constants (*_OFFSET).
// The product is rounded on its own (no contraction) so that the host
// read-back decodes identically.
template <int ST>
__device__ __forceinline__ float2 dec_ref(const StepParams &p, float2 own_prev,
                                          int i) {
  if (storage_local(ST))
    return make_float2(__fmul_rn(wgt(i), own_prev.x), __fmul_rn(wgt(i), own_prev.y));
  return make_float2(p.ref[0][wclass(i)], p.ref[1][wclass(i)]);
}

// The 19 populations of both components at the current time step, decoded
// to float32.
template <int PARITY, int ST>
__device__ __forceinline__ void load_pops(const StepParams &p, const Workspace &w,
                                          const Geo &g, float (&v1)[kQ],
                                          float (&v2)[kQ]) {
  using C = Codec2<ST>;
  const typename C::T2 *f = static_cast<const typename C::T2 *>(w.f);
  const long long nodes = p.ntiles * kTile, pairs = p.ntiles * kTilePairs;
  const int own = g.node(0, 0, 0);
  const float2 own_prev =
      storage_local(ST)
          ? __ldg(&w.rho_enc[(kChecked && !in_bounds(w.fault, own, nodes, kFaultRhoLoad)) ? 0 : own])
          : make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    // population i of node x: slot i at x (even), slot opp(i) at x - c_i (odd)
    const int slot = PARITY == 0 ? i : opp(i);
    const typename C::T2 *src =
        f + (PARITY == 0 ? g.pop_off(0, 0, 0) : g.pop_off(-cx(i), -cy(i), -cz(i)));
    if (kChecked && !in_bounds(w.fault, (src - f) + slot * kTile, pairs, kFaultPopLoad))
      src = f - slot * kTile;  // reads element 0
    const typename C::T2 raw = src[slot * kTile];
    const float2 v = C::dec(raw, dec_ref<ST>(p, own_prev, i));
    v1[i] = v.x;
    v2[i] = v.y;
  }
}

// Zeroth moment, summed in direction order; k_density and k_collide_stream
// share this order so both see bit-identical densities.
__device__ __forceinline__ float sum19(const float (&v)[kQ]) {
  float r = v[0];
#pragma unroll
  for (int i = 1; i < kQ; ++i) r += v[i];
  return r;
}

__device__ __forceinline__ void first_moment(const float (&v)[kQ],
                                             float (&j)[3]) {
  j[0] = j[1] = j[2] = 0.0f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    if (cx(i)) j[0] += cx(i) > 0 ? v[i] : -v[i];
    if (cy(i)) j[1] += cy(i) > 0 ? v[i] : -v[i];
    if (cz(i)) j[2] += cz(i) > 0 ? v[i] : -v[i];
  }
}

// A read-only load the compiler may neither merge with an earlier load of
// the same address nor hoist: keeps a value that is needed late from
// occupying a register from the start of the kernel.
__device__ __forceinline__ float2 ld_late(const float2 *ptr) {
  float2 v;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(ptr));
  return v;
}

// Where a pass finds the densities of the current step at x + (dx, dy, dz):
// `at` for the force stencil, `late` for the encoding reference of the
// *_LOCAL storages (a load the compiler keeps next to its use).
struct GlobalRho {  // the density array written by the density pass
  const float2 *__restrict__ rho;
  const Geo &g;
  long long nodes;   // tiled nodes (bounds-checked builds)
  unsigned *fault;
  __device__ __forceinline__ int idx(int dx, int dy, int dz) const {
    const int n = g.node(dx, dy, dz);
    return (kChecked && !in_bounds(fault, n, nodes, kFaultRhoLoad)) ? 0 : n;
  }
  __device__ __forceinline__ float2 at(int dx, int dy, int dz) const {
    return __ldg(&rho[idx(dx, dy, dz)]);
  }
  __device__ __forceinline__ float2 late(int dx, int dy, int dz) const {
    return ld_late(&rho[idx(dx, dy, dz)]);
  }
  // adhesion sources a_1 = G_ads,2 n_s,1 and a_2 (per-component fractions)
  const float *__restrict__ ads;
  const float *__restrict__ ads2;
  __device__ __forceinline__ int gidx(int dx, int dy, int dz) const {
    const int n = g.node(dx, dy, dz);
    return (kChecked && !in_bounds(fault, n, nodes, kFaultGeometry)) ? 0 : n;
  }
  __device__ __forceinline__ float a1(int dx, int dy, int dz) const {
    return __ldg(&ads[gidx(dx, dy, dz)]);
  }
  __device__ __forceinline__ float a2(int dx, int dy, int dz) const {
    return __ldg(&ads2[gidx(dx, dy, dz)]);
  }
};
__device__ __forceinline__ GlobalRho global_rho(const StepParams &p, const Workspace &w,
                                                const Geo &g) {
  return GlobalRho{w.rho, g, p.ntiles * kTile, w.fault, w.ads, w.ads2};
}

// Total force per unit mass of each component, F_tot,sigma / rho_sigma
// (Eqs. 3-5; rho_sigma cancels against the prefactor of Eqs. 3-4 and the
// density ratio of Eq. 5, so no division by a vanishing component density):
//   g_1 = -G S_2 + A_1 + F_ext / rho,   g_2 = -G S_1 - A_2 + F_ext / rho
// with S_sigma = sum_i w_i rho_sigma(x + c_i) c_i and A_sigma = sum_i w_i
// a_sigma(x + c_i) c_i, a_sigma = G_ads,2 n_s,sigma (G_ads,1 = -G_ads,2,
// Table 1; the indicator of Eq. 4 is the component's own fraction).  With
// one fraction for both (PC = false) A_1 = A_2.  Opposite directions are
// summed as pairs, so a uniform field gives exactly zero.
template <bool PC, typename RS>
__device__ __forceinline__ void force_per_mass(const StepParams &p, const RS &rs,
                                               const Workspace &w, const Geo &g,
                                               float rho_tot, float (&g1)[3],
                                               float (&g2)[3]) {
  float s1[3] = {0.f, 0.f, 0.f}, s2[3] = {0.f, 0.f, 0.f};
  float sa[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 1; i <= 9; ++i) {
    const float2 rp = rs.at(cx(i), cy(i), cz(i));
    const float2 rm = rs.at(-cx(i), -cy(i), -cz(i));
    const float ap = rs.a1(cx(i), cy(i), cz(i));
    const float am = rs.a1(-cx(i), -cy(i), -cz(i));
    const float d1 = wgt(i) * (rp.x - rm.x);
    const float d2 = wgt(i) * (rp.y - rm.y);
    const float da = wgt(i) * (ap - am);
    float db = 0.0f;
    if (PC) db = wgt(i) * (rs.a2(cx(i), cy(i), cz(i)) - rs.a2(-cx(i), -cy(i), -cz(i)));
    if (cx(i)) { s1[0] += cx(i) > 0 ? d1 : -d1; s2[0] += cx(i) > 0 ? d2 : -d2; sa[0] += cx(i) > 0 ? da : -da; if (PC) sb[0] += cx(i) > 0 ? db : -db; }
    if (cy(i)) { s1[1] += cy(i) > 0 ? d1 : -d1; s2[1] += cy(i) > 0 ? d2 : -d2; sa[1] += cy(i) > 0 ? da : -da; if (PC) sb[1] += cy(i) > 0 ? db : -db; }
    if (cz(i)) { s1[2] += cz(i) > 0 ? d1 : -d1; s2[2] += cz(i) > 0 ? d2 : -d2; sa[2] += cz(i) > 0 ? da : -da; if (PC) sb[2] += cz(i) > 0 ? db : -db; }
  }
  const float inv_rho = 1.0f / rho_tot;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float fe = p.F[d] * inv_rho;
    g1[d] = -p.G * s2[d] + sa[d] + fe;
    g2[d] = -p.G * s1[d] - (PC ? sb[d] : sa[d]) + fe;
  }
}

// Reservoir face holding node (x, y, z), -1 if none; the higher face wins.
__device__ __forceinline__ int res_face(const StepParams &p, int x, int y,
                                        int z) {
  const int *L = p.res.layers;
  int face = -1;
  if (L[0] && x < L[0]) face = 0;
  if (L[1] && x >= p.nx - L[1]) face = 1;
  if (L[2] && y < L[2]) face = 2;
  if (L[3] && y >= p.ny - L[3]) face = 3;
  if (L[4] && z < L[4]) face = 4;
  if (L[5] && z >= p.nz - L[5]) face = 5;
  return face;
}

// rho_res of component s on face `face` (selects, no indexed parameter load).
__device__ __forceinline__ float res_rho(const StepParams &p, int face, int s) {
  float r = p.res.rho[0][s];
#pragma unroll
  for (int k = 1; k < kFaces; ++k) r = face == k ? p.res.rho[k][s] : r;
  return r;
}

// Does the block's box [xlo,xhi] x [ylo,yhi] x [zlo,zhi] hold a node inside
// a reservoir?  Uniform over the block, known before any load.
__device__ __forceinline__ bool box_in_reservoir(const StepParams &p, int xlo,
                                                 int xhi, int ylo, int yhi,
                                                 int zlo, int zhi) {
  if (!p.res.any) return false;
  const int *L = p.res.layers;
  return (L[0] && xlo < L[0]) || (L[1] && xhi >= p.nx - L[1]) ||
         (L[2] && ylo < L[2]) || (L[3] && yhi >= p.ny - L[3]) ||
         (L[4] && zlo < L[4]) || (L[5] && zhi >= p.nz - L[5]);
}

// Prescribed velocity component d of face `face` (selects).
__device__ __forceinline__ float res_u(const StepParams &p, int face, int d) {
  float u = p.res.u[0][d];
#pragma unroll
  for (int k = 1; k < kFaces; ++k) u = face == k ? p.res.u[k][d] : u;
  return u;
}

// A node inside a reservoir holds the prescribed equilibrium: at rest for a
// density reservoir, at the face's velocity for velocity boundary cells.
// Only blocks whose box meets a reservoir (`maybe`, block-uniform) look.
__device__ __forceinline__ void reservoir_state(const StepParams &p, bool maybe,
                                                int x, int y, int z,
                                                float (&v1)[kQ], float (&v2)[kQ]) {
  if (!maybe) return;
  const int face = res_face(p, x, y, z);
  if (face >= 0) {
    const float r1 = res_rho(p, face, 0), r2 = res_rho(p, face, 1);
    if (p.res.moving) {
      const float ux = res_u(p, face, 0), uy = res_u(p, face, 1), uz = res_u(p, face, 2);
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        v1[i] = res_feq(i, r1, ux, uy, uz);
        v2[i] = res_feq(i, r2, ux, uy, uz);
      }
    } else {
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        v1[i] = wgt(i) * r1;
        v2[i] = wgt(i) * r2;
      }
    }
  }
}

// Store the post-collision pair (both components) of direction i; it
// becomes the pair of direction i of node x + c_i at t + 1.  Encoding
// reference: w_i times the destination's density at this step (*_LOCAL;
// rho_s for the rest population, the density pass's value otherwise), or the
// constants w_i rho0_sigma (*_OFFSET).
template <int PARITY, int ST, typename RS, bool CS = false>
__device__ __forceinline__ void put2(const StepParams &p, const Workspace &w,
                                     const Geo &g, const RS &rs, int i, float o1,
                                     float o2, float r1, float r2) {
  using C = Codec2<ST>;
  typename C::T2 *f = static_cast<typename C::T2 *>(w.f);
  // encoding reference times the codec's scale (exact)
  float2 ref = make_float2(p.ref[0][wclass(i)] * C::kScale, p.ref[1][wclass(i)] * C::kScale);
  if (storage_local(ST)) {
    const float2 rd = i == 0 ? make_float2(r1, r2) : rs.late(cx(i), cy(i), cz(i));
    const float ws = wgt(i) * C::kScale;
    ref = make_float2(__fmul_rn(ws, rd.x), __fmul_rn(ws, rd.y));
  }
  const typename C::T2 e = C::enc_s(o1, o2, ref);
  const int slot = PARITY == 0 ? opp(i) : i;
  typename C::T2 *dst = f + (PARITY == 0 ? g.pop_off(0, 0, 0) : g.pop_off(cx(i), cy(i), cz(i)));
  if (!kChecked ||
      in_bounds(w.fault, (dst - f) + slot * kTile, p.ntiles * kTilePairs, kFaultPopStore))
  {
    if (CS)
      __stcs(&dst[slot * kTile], e);  // streaming: evict first from the caches
    else
      dst[slot * kTile] = e;
  }
}

// Eq. 1 for both components: (1 - n_s)[f_i - (f_i - f^eq_i)/tau] +
// n_s f_opp(i) with f^eq of Eq. A.3 at (rho_s, u_s), computed for opposite
// pairs at once.  The rest population's equilibrium is taken as rho_s minus
// the other 18 (sum_i f^eq_i = rho_s holds exactly for Eq. A.3 on D3Q19),
// which keeps the rounding of the float weights from leaking mass step after
// step.  The relaxation weight b = (1 - n_s) / tau is folded into the
// equilibrium: B_i = b f^eq_i = (b w_i rho_s)[1 - 1.5 u.u + 4.5 (c_i.u)^2
// +- 3 c_i.u], so each population costs two fused multiply-adds on top of B_i.
struct Relax {
  float a, base, br, br18, br36, moving, nsx;
  __device__ __forceinline__ Relax(float om, float ns_s, float rho_s, const float (&u)[3]) {
    nsx = ns_s;
    a = (1.0f - nsx) * (1.0f - om);
    const float b = (1.0f - nsx) * om;
    base = 1.0f - 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    br = b * rho_s;
    br18 = br * (1.0f / 18.0f);
    br36 = br * (1.0f / 36.0f);
    moving = 0.0f;  // sum of B_i over the 18 moving directions
  }
  // post-collision values of the opposite pair (i, i + 9) from their
  // pre-collision values vi, vj
  __device__ __forceinline__ void pair_s(int i, const float (&u)[3], float vi, float vj,
                                         float &out_i, float &out_j) {
    const float cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
    const float bw = wgt(i) == (1.0f / 18.0f) ? br18 : br36;
    const float even = bw * fmaf(4.5f * cu, cu, base);
    const float odd = (3.0f * bw) * cu;
    const float B_i = even + odd, B_j = even - odd;
    moving += B_i + B_j;
    out_i = fmaf(a, vi, fmaf(nsx, vj, B_i));
    out_j = fmaf(a, vj, fmaf(nsx, vi, B_j));
  }
  __device__ __forceinline__ void pair(int i, const float (&u)[3], const float (&v)[kQ],
                                       float &out_i, float &out_j) {
    pair_s(i, u, v[i], v[i + 9], out_i, out_j);
  }
  // post-collision rest population: B_0 = b rho_s - sum of the moving B_i
  __device__ __forceinline__ float rest_s(float v0) const {
    return fmaf(a + nsx, v0, br - moving);
  }
  __device__ __forceinline__ float rest(const float (&v)[kQ]) const { return rest_s(v[0]); }
};

template <int PARITY, int ST, typename RS, bool CS = false>
__device__ __forceinline__ void collide_put2(const StepParams &p, const Workspace &w,
                                             const Geo &g, const RS &rs,
                                             const float (&v1)[kQ],
                                             const float (&v2)[kQ], float r1,
                                             float r2, const float (&u1)[3],
                                             const float (&u2)[3], float ns1,
                                             float ns2) {
  Relax c1(p.omega[0], ns1, r1, u1), c2(p.omega[1], ns2, r2, u2);
#pragma unroll
  for (int i = 1; i <= 9; ++i) {
    float o1i, o1j, o2i, o2j;
    c1.pair(i, u1, v1, o1i, o1j);
    c2.pair(i, u2, v2, o2i, o2j);
    put2<PARITY, ST, RS, CS>(p, w, g, rs, i, o1i, o2i, r1, r2);
    put2<PARITY, ST, RS, CS>(p, w, g, rs, i + 9, o1j, o2j, r1, r2);
  }
  put2<PARITY, ST, RS, CS>(p, w, g, rs, 0, c1.rest(v1), c2.rest(v2), r1, r2);
}

// Moments, forces, equilibrium velocity and collision of node (x, y, z)
// given its neighbourhood g and the source of the step's densities.
// collide_loaded starts from the node's 38 populations already decoded (and
// replaced by the prescribed state inside a reservoir).
template <int PARITY, int ST, bool PC, typename RS, bool CS = false>
__device__ __forceinline__ void collide_loaded(const StepParams &p, const Workspace &w,
                                               const Geo &g, const RS &rs,
                                               const float (&f1)[kQ],
                                               const float (&f2)[kQ]) {
  const float r1 = sum19(f1), r2 = sum19(f2);
  float j1[3], j2[3];
  first_moment(f1, j1);
  first_moment(f2, j2);

  float g1[3], g2[3];
  force_per_mass<PC>(p, rs, w, g, r1 + r2, g1, g2);

  // Eq. 6: common velocity sum_s j_s/tau_s / sum_s rho_s/tau_s, then the
  // Shan-Chen shift tau_s F_tot,s / rho_s = tau_s g_s.
  const float inv_den = 1.0f / (r1 * p.omega[0] + r2 * p.omega[1]);
  float u1[3], u2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float uc = (j1[d] * p.omega[0] + j2[d] * p.omega[1]) * inv_den;
    u1[d] = uc + p.tau[0] * g1[d];
    u2[d] = uc + p.tau[1] * g2[d];
  }

  int own = g.node(0, 0, 0);
  if (!in_bounds(w.fault, own, p.ntiles * kTile, kFaultGeometry)) own = 0;
  const float ns1 = w.ns[own];
  const float ns2 = PC ? w.ns2[own] : ns1;
  collide_put2<PARITY, ST, RS, CS>(p, w, g, rs, f1, f2, r1, r2, u1, u2, ns1, ns2);
}

template <int PARITY, int ST, bool PC, typename RS>
__device__ __forceinline__ void collide_node(const StepParams &p, const Workspace &w,
                                             const Geo &g, const RS &rs,
                                             bool maybe_res, int x, int y, int z) {
  float f1[kQ], f2[kQ];
  load_pops<PARITY, ST>(p, w, g, f1, f2);
  reservoir_state(p, maybe_res, x, y, z, f1, f2);
  collide_loaded<PARITY, ST, PC>(p, w, g, rs, f1, f2);
}

template <int PARITY, int ST, bool PC, bool CS = false>
__device__ __forceinline__ void collide_body(const StepParams &p,
                                             const Workspace &w, bool maybe_res,
                                             int x, int y, int z) {
  const Geo g = make_geo(p, x, y, z);
  float f1[kQ], f2[kQ];
  load_pops<PARITY, ST>(p, w, g, f1, f2);
  reservoir_state(p, maybe_res, x, y, z, f1, f2);
  collide_loaded<PARITY, ST, PC, GlobalRho, CS>(p, w, g, global_rho(p, w, g), f1, f2);
}


// Launch shapes of the passes: a block is 32 x by x bz threads (one node
// each) and minb is the number of blocks per SM its register budget is sized
// for.  Shape 0 of each pass is the default; the autotuner picks among the
// others per lattice size and storage.
struct Shape {
  int by, bz, minb;
  bool cs = false;  // populations stored with the streaming (evict-first) policy
};
__host__ __device__ constexpr Shape density_shape(int cfg) {
  return cfg == 1 ? Shape{8, 1, 1} : cfg == 2 ? Shape{4, 1, 1} : Shape{4, 2, 1};
}
// Shapes of the prefetching fused pass (k_collide_pipe): block 32 x by,
// blocks per SM, planes per block (zc) and shared-memory buffers (nb, so
// nb - 1 planes are in flight).
struct PipeCfg {
  int by, minb_even, minb_odd, minb_even_local, minb_odd_local, zc, nb;
  bool ring;  // neighbour densities and adhesion sources also staged in
              // shared memory (a five-plane ring filled by the block)
  bool cs;    // streaming stores
};
// Measured on the 256^3 electrode: one plane in flight (nb = 2) beats two
// (nb = 3, fewer blocks fit), and the best shapes are 8 rows for even steps
// and 2 rows at 8 blocks per SM for odd steps.  Staging the neighbour
// densities in a ring as well (shape 8) helps the half-offset odd step by
// ~3 % and the local 16-bit even step by 6 %, and slows the float32 one (the
// per-plane barrier); with streaming stores (shape 9) the local odd step
// drops from 0.93 to 0.80 ms.
__host__ __device__ constexpr PipeCfg pipe_cfg(int cfg) {
  return cfg == 6   ? PipeCfg{8, 2, 2, 2, 2, 16, 2, false, false}
         : cfg == 7 ? PipeCfg{2, 10, 8, 8, 6, 16, 2, false, false}
         : cfg == 8 ? PipeCfg{2, 10, 8, 8, 6, 16, 2, true, false}
         : cfg == 9 ? PipeCfg{2, 10, 8, 8, 6, 16, 2, true, true}
                    : PipeCfg{4, 5, 4, 4, 3, 8, 2, false, false};
}
// Shared memory of a prefetching block: population buffers, then (ring)
// five planes of (by + 2) x 34 density pairs and adhesion sources.
constexpr int kPipeRingPlanes = 5, kPipeRingCols = kTile + 2;
__host__ __device__ constexpr int pipe_smem_bytes(int cfg, int pair_bytes, bool pc) {
  return pipe_cfg(cfg).nb * kQ * kTile * pipe_cfg(cfg).by * pair_bytes +
         (pipe_cfg(cfg).ring ? kPipeRingPlanes * (pipe_cfg(cfg).by + 2) * kPipeRingCols *
                                   (8 + 4 + (pc ? 4 : 0))
                             : 0);
}

// Neighbour densities and adhesion sources from the shared-memory ring of a
// prefetching block: row pointers of the node's ring row in planes z - 1,
// z, z + 1 and the node's column.
struct SmemStencil {
  const float2 *rho[3];
  const float *a[3];
  const float *b[3];
  int c;
  __device__ __forceinline__ float2 at(int dx, int dy, int dz) const {
    return rho[dz + 1][dy * kPipeRingCols + c + dx];
  }
  __device__ __forceinline__ float2 late(int dx, int dy, int dz) const {
    return at(dx, dy, dz);
  }
  __device__ __forceinline__ float a1(int dx, int dy, int dz) const {
    return a[dz + 1][dy * kPipeRingCols + c + dx];
  }
  __device__ __forceinline__ float a2(int dx, int dy, int dz) const {
    return b[dz + 1][dy * kPipeRingCols + c + dx];
  }
};
__host__ __device__ constexpr Shape pipe_shape(int parity, bool local, int cfg) {
  return Shape{pipe_cfg(cfg).by, 1,
               parity == 0 ? (local ? pipe_cfg(cfg).minb_even_local : pipe_cfg(cfg).minb_even)
                           : (local ? pipe_cfg(cfg).minb_odd_local : pipe_cfg(cfg).minb_odd),
               pipe_cfg(cfg).cs};
}
// The odd step keeps one address per neighbour offset and the *_LOCAL
// storages also hold the destination densities for encoding: both get more
// registers per thread (the local odd shape 2 trades occupancy for a budget
// of 170 registers, which needs no spill).  Shape 4 stores with the
// streaming policy (float32 odd step 1.05 -> 0.95 ms in the plain kernel).
__host__ __device__ constexpr Shape collide_shape(int parity, bool local, int cfg) {
  return cfg >= kCollidePipeFirst ? pipe_shape(parity, local, cfg)
         : cfg == 4 ? (local ? Shape{4, 1, 3, true} : Shape{4, 2, 2, true})
         : parity == 0
             ? (local ? (cfg == 1 ? Shape{8, 1, 2} : cfg == 2 ? Shape{4, 1, 4}
                         : cfg == 3 ? Shape{2, 4, 2} : Shape{4, 2, 2})
                      : (cfg == 1 ? Shape{8, 1, 3} : cfg == 2 ? Shape{4, 1, 6}
                         : cfg == 3 ? Shape{2, 4, 3} : Shape{4, 2, 3}))
             : (local ? (cfg == 1 ? Shape{4, 2, 2} : cfg == 2 ? Shape{4, 1, 3}
                         : cfg == 3 ? Shape{2, 2, 4} : Shape{4, 1, 4})
                      : (cfg == 1 ? Shape{4, 2, 2} : cfg == 2 ? Shape{8, 1, 2}
                         : cfg == 3 ? Shape{2, 2, 5} : Shape{4, 1, 5}));
}
template <int CFG>
struct DensityShape {
  static constexpr Shape s = density_shape(CFG);
  static constexpr int threads = kTile * s.by * s.bz;
};
template <int PARITY, int ST, int CFG>
struct CollideShape {
  static constexpr Shape s = collide_shape(PARITY, storage_local(ST), CFG);
  static constexpr int threads = kTile * s.by * s.bz;
};
constexpr int kFieldsBY = 4, kFieldsBZ = 2;

// Does the block's box hold a node inside a reservoir?  Block-uniform.
template <int BY, int BZ>
__device__ __forceinline__ bool block_in_reservoir(const StepParams &p) {
  const int xlo = blockIdx.x * kTile, ylo = blockIdx.y * BY, zlo = blockIdx.z * BZ;
  return box_in_reservoir(p, xlo, min(xlo + kTile, p.nx) - 1, ylo,
                          min(ylo + BY, p.ny) - 1, zlo, min(zlo + BZ, p.nz) - 1);
}

template <int BY, int BZ>
__device__ __forceinline__ void block_coords(int &x, int &y, int &z) {
  x = blockIdx.x * kTile + threadIdx.x;
  y = blockIdx.y * BY + threadIdx.y;
  z = blockIdx.z * BZ + threadIdx.z;
}

template <int PARITY, int ST, int CFG>
__global__ void __launch_bounds__(DensityShape<CFG>::threads)
    k_density(StepParams p, Workspace w) {
  constexpr Shape S = DensityShape<CFG>::s;
  int x, y, z;
  block_coords<S.by, S.bz>(x, y, z);
  const bool maybe_res = block_in_reservoir<S.by, S.bz>(p);
  if (x >= p.nx || y >= p.ny || z >= p.nz) return;
  const Geo g = make_geo(p, x, y, z);
  float v1[kQ], v2[kQ];
  load_pops<PARITY, ST>(p, w, g, v1, v2);
  reservoir_state(p, maybe_res, x, y, z, v1, v2);
  const int own = g.node(0, 0, 0);
  if (in_bounds(w.fault, own, p.ntiles * kTile, kFaultRhoStore))
    w.rho[own] = make_float2(sum19(v1), sum19(v2));
}

// ---- fused pass with prefetch ----
// Shapes kCollidePipeFirst.. of the fused pass: each block owns 32 x by
// nodes of a run of planes and walks the run plane by plane; every thread
// copies the populations of its node in the next plane into shared memory
// (cp.async, two buffers, the thread's own slots only, so no barrier) while
// it collides the current plane.  The loads of one node overlap the
// arithmetic of the one before without holding registers; the arithmetic is
// that of k_collide_stream, so the results are bit-identical.
template <typename T>
__device__ __forceinline__ void cp_async(T *smem, const T *gmem) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async copies 4 or 8 bytes here");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem),
               "n"((int)sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}


// The fused pass of one block of a prefetching shape: x-tile bx, rows
// [by0 * by, by0 * by + by) and the run of planes [bz * zc, bz * zc + zc)
// of lattice (p, w).
template <int PARITY, int ST, bool PC, int CFG>
__device__ __forceinline__ void pipe_block(const StepParams &p, const Workspace &w, int bx,
                                           int by0, int bz) {
  using C = Codec2<ST>;
  using T2 = typename C::T2;
  constexpr Shape S = CollideShape<PARITY, ST, CFG>::s;
  constexpr int NT = kTile * S.by;
  constexpr PipeCfg P = pipe_cfg(CFG);
  constexpr int ZC = P.zc, NB = P.nb, R = S.by + 2, RC = kPipeRingCols;
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  T2(*buf)[kQ][NT] = reinterpret_cast<T2(*)[kQ][NT]>(pipe_smem);  // [NB][kQ][NT]
  // ring: [5][R][RC] density pairs, then adhesion sources a_1 (and a_2)
  float2 *ring_rho = reinterpret_cast<float2 *>(pipe_smem + NB * kQ * NT * sizeof(T2));
  float *ring_a = reinterpret_cast<float *>(ring_rho + kPipeRingPlanes * R * RC);
  float *ring_b = ring_a + kPipeRingPlanes * R * RC;
  const int tid = threadIdx.y * kTile + threadIdx.x;
  const int x = bx * kTile + threadIdx.x, y = by0 * S.by + threadIdx.y;
  const int z0 = bz * ZC, zend = min(z0 + ZC, p.nz);
  const int xlo = bx * kTile, ylo = by0 * S.by;
  const bool maybe_res = box_in_reservoir(p, xlo, min(xlo + kTile, p.nx) - 1, ylo,
                                          min(ylo + S.by, p.ny) - 1, z0, zend - 1);
  const bool active = x < p.nx && y < p.ny;
  // Without the ring no thread reads another's shared memory and idle
  // threads may leave; with it every thread fills the ring and meets the
  // per-plane barrier.
  if (z0 >= zend || (!P.ring && !active)) return;
  const T2 *f = static_cast<const T2 *>(w.f);
  const long long pairs = p.ntiles * kTilePairs, nodes = p.ntiles * kTile;
  auto prefetch = [&](int z, int b) {
    if (!active) return;
    const Geo g = make_geo(p, x, y, z);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int slot = PARITY == 0 ? i : opp(i);
      const T2 *src = f + (PARITY == 0 ? g.pop_off(0, 0, 0) : g.pop_off(-cx(i), -cy(i), -cz(i)));
      if (kChecked && !in_bounds(w.fault, (src - f) + slot * kTile, pairs, kFaultPopLoad))
        src = f - slot * kTile;
      cp_async(&buf[b][i][tid], src + slot * kTile);
    }
  };
  // ring plane of z (z0 - 1 <= z <= zend): rows y0 - 1 .. y0 + by, columns
  // x0 - 1 .. x0 + 32, periodic
  auto fill_ring = [&](int z) {
    const int slot = (z - z0 + 1) % kPipeRingPlanes;
    const int zw = z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z);
    for (int e = tid; e < R * RC; e += NT) {
      const int r = e / RC, c = e % RC;
      int xw = xlo + c - 1, yw = ylo + r - 1;
      xw = xw < 0 ? xw + p.nx : (xw >= p.nx ? xw % p.nx : xw);
      yw = yw < 0 ? yw + p.ny : (yw >= p.ny ? yw % p.ny : yw);
      long long n = ((long long)(zw * p.ny + yw) * p.ntx + xw / kTile) * kTile + xw % kTile;
      if (kChecked && !in_bounds(w.fault, n, nodes, kFaultRhoLoad)) n = 0;
      const int k = (slot * R + r) * RC + c;
      cp_async(&ring_rho[k], &w.rho[n]);
      cp_async(&ring_a[k], &w.ads[n]);
      if (PC) cp_async(&ring_b[k], &w.ads2[n]);
    }
  };
  if constexpr (!P.ring) {
    // NB - 1 planes in flight; one commit group per plane (empty past the end)
#pragma unroll
    for (int d = 0; d + 1 < NB; ++d) {
      if (z0 + d < zend) prefetch(z0 + d, d);
      cp_async_commit();
    }
  } else {
    prefetch(z0, 0);
    fill_ring(z0 - 1);
    fill_ring(z0);
    fill_ring(z0 + 1);
    cp_async_commit();
  }
  for (int z = z0; z < zend; ++z) {
    const int b = (z - z0) % NB;
    if constexpr (!P.ring) {
      const int zp = z + NB - 1;
      // buffer (zp - z0) % NB was consumed by the previous plane
      if (zp < zend) prefetch(zp, (zp - z0) % NB);
      cp_async_commit();
      cp_async_wait<NB - 1>();  // the group of plane z is complete
    } else {
      // next plane's populations and the ring plane after it; the ring slot
      // refilled here was last read two planes ago, before the previous
      // barrier
      if (z + 1 < zend) prefetch(z + 1, (z + 1 - z0) % NB);
      if (z + 2 <= zend) fill_ring(z + 2);
      cp_async_commit();
      cp_async_wait<1>();   // this thread's copies for plane z are complete
      __syncthreads();      // and every thread's ring copies too
    }
    if (!active) continue;
    const Geo g = make_geo(p, x, y, z);
    const int own = g.node(0, 0, 0);
    const float2 own_prev =
        storage_local(ST)
            ? __ldg(&w.rho_enc[(kChecked && !in_bounds(w.fault, own, nodes, kFaultRhoLoad)) ? 0 : own])
            : make_float2(0.f, 0.f);
    float f1[kQ], f2[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float2 v = C::dec(buf[b][i][tid], dec_ref<ST>(p, own_prev, i));
      f1[i] = v.x;
      f2[i] = v.y;
    }
    reservoir_state(p, maybe_res, x, y, z, f1, f2);
    if constexpr (!P.ring) {
      collide_loaded<PARITY, ST, PC, GlobalRho, S.cs>(p, w, g, global_rho(p, w, g), f1, f2);
    } else {
      SmemStencil st;
      const int r = threadIdx.y + 1;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int k = (((z - 1 + d) - z0 + 1) % kPipeRingPlanes * R + r) * RC;
        st.rho[d] = ring_rho + k;
        st.a[d] = ring_a + k;
        st.b[d] = ring_b + k;
      }
      st.c = threadIdx.x + 1;
      collide_loaded<PARITY, ST, PC, SmemStencil, S.cs>(p, w, g, st, f1, f2);
    }
  }
}

template <int PARITY, int ST, bool PC, int CFG>
__global__ void __launch_bounds__(CollideShape<PARITY, ST, CFG>::threads,
                                  CollideShape<PARITY, ST, CFG>::s.minb)
    k_collide_pipe(StepParams p, Workspace w) {
  pipe_block<PARITY, ST, PC, CFG>(p, w, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int PARITY, int ST, int CFG, bool PC>
__global__ void __launch_bounds__(CollideShape<PARITY, ST, CFG>::threads,
                                  CollideShape<PARITY, ST, CFG>::s.minb)
    k_collide_stream(StepParams p, Workspace w) {
  constexpr Shape S = CollideShape<PARITY, ST, CFG>::s;
  int x, y, z;
  block_coords<S.by, S.bz>(x, y, z);
  const bool maybe_res = block_in_reservoir<S.by, S.bz>(p);
  if (x >= p.nx || y >= p.ny || z >= p.nz) return;
  collide_body<PARITY, ST, PC, S.cs>(p, w, maybe_res, x, y, z);
}

// Macroscopic fields of the current state into the linear staging planes:
// rho_1, rho_2, u_macro (Eq. 7) x, y, z, p (Eq. A.6).
template <int PARITY, int ST, bool PC>
__global__ void __launch_bounds__(kTile * kFieldsBY * kFieldsBZ)
    k_fields(StepParams p, Workspace w) {
  int x, y, z;
  block_coords<kFieldsBY, kFieldsBZ>(x, y, z);
  const bool maybe_res = block_in_reservoir<kFieldsBY, kFieldsBZ>(p);
  if (x >= p.nx || y >= p.ny || z >= p.nz) return;
  const Geo g = make_geo(p, x, y, z);
  float f1[kQ], f2[kQ];
  load_pops<PARITY, ST>(p, w, g, f1, f2);
  reservoir_state(p, maybe_res, x, y, z, f1, f2);
  const float r1 = sum19(f1), r2 = sum19(f2);
  float j1[3], j2[3];
  first_moment(f1, j1);
  first_moment(f2, j2);
  float g1[3], g2[3];
  const float rho = r1 + r2;
  force_per_mass<PC>(p, global_rho(p, w, g), w, g, rho, g1, g2);
  int own = g.node(0, 0, 0);
  if (!in_bounds(w.fault, own, p.ntiles * kTile, kFaultGeometry)) own = 0;
  const float fluid = 1.0f - w.ns[own];
  const float fluid2 = PC ? 1.0f - w.ns2[own] : fluid;
  const long long L = p.nlin;
  const long long n = x + (long long)p.nx * (y + (long long)p.ny * z);
  if (!in_bounds(w.fault, n, L, kFaultStage)) return;
  w.stage[n] = r1;
  w.stage[L + n] = r2;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (PC) {
      const float m = fluid * (j1[d] + 0.5f * r1 * g1[d]) +
                      fluid2 * (j2[d] + 0.5f * r2 * g2[d]);
      w.stage[(2 + d) * L + n] = m / rho;
    } else {
      const float m = (j1[d] + 0.5f * r1 * g1[d]) + (j2[d] + 0.5f * r2 * g2[d]);
      w.stage[(2 + d) * L + n] = fluid * m / rho;
    }
  }
  w.stage[5 * L + n] = (rho + p.G * r1 * r2) * (1.0f / 3.0f);
}

// Tiled node index of linear node n = x + nx (y + ny z).
__device__ __forceinline__ long long tiled_of_linear(const StepParams &p,
                                                     long long n) {
  const int x = (int)(n % p.nx);
  const long long yz = n / p.nx;
  return (yz * p.ntx + x / kTile) * kTile + x % kTile;
}

// f_i = w_i rho_sigma at rest.  *_LOCAL storages take the initial
// densities as the previous densities of time 0.
template <int ST>
__global__ void k_init_equilibrium(StepParams p, Workspace w,
                                   const float *__restrict__ rho1,
                                   const float *__restrict__ rho2) {
  using C = Codec2<ST>;
  const long long N = (long long)p.nx * p.ny * p.nz;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const long long tn = tiled_of_linear(p, n);
    if (!in_bounds(w.fault, tn, p.ntiles * kTile, kFaultPopStore)) continue;
    typename C::T2 *b = static_cast<typename C::T2 *>(w.f) + (tn / kTile) * kTilePairs + tn % kTile;
    const float r1 = rho1[n], r2 = rho2[n];
    if (storage_local(ST)) w.rho_enc[tn] = make_float2(r1, r2);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      float2 ref = make_float2(p.ref[0][wclass(i)], p.ref[1][wclass(i)]);
      if (storage_local(ST)) ref = make_float2(__fmul_rn(wgt(i), r1), __fmul_rn(wgt(i), r2));
      b[i * kTile] = C::enc(__fmul_rn(wgt(i), r1), __fmul_rn(wgt(i), r2), ref);
    }
  }
}

// ---- wavefront step: both passes in one persistent launch ----
// The lattice is cut into items: tile T (32 x by nodes of one plane) of
// group g, g = 0 .. nz + lag - 1, numbered group-major and taken by the
// blocks in the order of an atomic ticket.  Item (g, T)
//   - copies the populations of plane q = g - lag of T (if q >= 0) and of
//     plane d(g) = (g - 1) mod nz of T (if g < nz) into shared memory,
//   - waits until the densities of planes q - 1 .. q + 1 of T and of its
//     eight in-plane neighbour tiles are published, then collides and
//     streams plane q of T exactly as k_collide_stream does,
//   - sums the populations of plane d(g) into the density array and
//     publishes them: after a block barrier one thread sets the flag of
//     (d(g), T) to the launch's epoch with a release store.
// The densities a collision of plane q needs come from groups q .. q + 2,
// all before g when lag >= 3, so an item waits only on items with smaller
// tickets; those are held by blocks that are already running, so the launch
// cannot deadlock for any number of resident blocks (every wait is bounded
// all the same, and the launch is cooperative, so every block is resident
// anyway).  The populations of plane q were read from DRAM by the density
// part lag - 1 groups earlier (a group is one plane of the lattice, 10 MB at
// 256^2 in float32) and the collision finds them in L2: one step moves its
// populations through DRAM once instead of twice.  In-place AA streaming
// stays race-free: the collision of node n touches only the slots holding
// n's own populations, whose density part has finished reading them before
// n's flag is set.
struct WaveCfg {
  int by, minb, minb_local;
};
__host__ __device__ constexpr WaveCfg wave_cfg(int cfg) {
  return cfg == 2 ? WaveCfg{2, 8, 6} : cfg == 3 ? WaveCfg{8, 2, 2} : WaveCfg{4, 4, 3};
}
template <int ST, int CFG>
struct WaveShape {
  static constexpr WaveCfg c = wave_cfg(CFG);
  static constexpr int threads = kTile * c.by;
  static constexpr int minb = storage_local(ST) ? c.minb_local : c.minb;
};
struct WaveArgs {
  unsigned items;       // (nz + lag) * tp
  int tp;               // tiles per plane: ntx * ceil(ny / by)
  int lag;
  unsigned spin_limit;  // polls of one flag before a wait gives up (a few
                        // seconds at the default with the back-off); the item
                        // then goes on and the fault word records kFaultWait
  long long hold;       // a flag the launch leaves unpublished, -1: none
                        // (tests of the failure path)
};

// Flags are polled with relaxed loads, served by L2, so polling leaves the
// SM's L1 alone (an acquire would drop it, and with it the stencil's cached
// densities and geometry, once per poll).  A flag is set by a release store
// after the tile's density stores, so once a poll sees the epoch those
// densities are in L2; the loads that read them are issued after the poll
// returned, and no SM caches a line of a tile's densities in L1 before that
// tile's flag is set in this launch (each 128-byte line belongs to one
// tile, and L1 is invalidated between launches), so they miss L1 the first
// time and read L2.
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *ptr) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ptr) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned *ptr, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(ptr), "r"(v) : "memory");
}

// A wavefront wait that ran out: the fault word records it (and the mapped
// host word, when there is one), and wave[3] names the launch, so that the
// launch's other waits give up at once while later launches wait as usual.
__device__ __forceinline__ void wave_fault(const Workspace &w, unsigned epoch) {
  atomicOr(w.fault, kFaultWait);
  *(volatile unsigned *)&w.wave[3] = epoch;
  if (w.fault_host) *(volatile unsigned *)w.fault_host = kFaultWait;
}

// Densities written earlier in the same launch by other blocks, read after
// their flags (see above), cached in L1 for the stencil.
struct WaveRho : GlobalRho {
  __device__ __forceinline__ float2 at(int dx, int dy, int dz) const {
    return __ldca(&rho[idx(dx, dy, dz)]);
  }
  __device__ __forceinline__ float2 late(int dx, int dy, int dz) const {
    const float2 *ptr = &rho[idx(dx, dy, dz)];
    float2 v;
    asm volatile("ld.global.ca.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(ptr));
    return v;
  }
};

// One wavefront item: ticket k of the launch's lattice (p, w).  buf is the
// block's two population buffers (this thread's own slots: [b][i][tid]),
// epoch the lattice's launch epoch, hold a flag left unpublished (-1: none;
// failure-path tests).  Ends after a block barrier with the tile's densities
// stored and published and the buffers free.
template <int PARITY, int ST, bool PC, int BY>
__device__ __forceinline__ void wave_tile_item(const StepParams &p, const Workspace &w,
                                               unsigned k, const WaveArgs &a, long long hold,
                                               typename Codec2<ST>::T2 (*buf)[kQ][kTile * BY],
                                               unsigned epoch) {
  using C = Codec2<ST>;
  using T2 = typename C::T2;
  const int tid = threadIdx.y * kTile + threadIdx.x;
  unsigned *ctl = w.wave, *flag = w.wave + kWaveCtlWords;
  const T2 *f = static_cast<const T2 *>(w.f);
  const long long pairs = p.ntiles * kTilePairs, nodes = p.ntiles * kTile;
  const long long nflags = (long long)p.nz * a.tp;
  const int nty = a.tp / p.ntx;
  // populations of node (x, y, z) into buffer b (this thread's own slots)
  auto copy = [&](int x, int y, int z, int b) {
    const Geo g = make_geo(p, x, y, z);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int slot = PARITY == 0 ? i : opp(i);
      const T2 *src = f + (PARITY == 0 ? g.pop_off(0, 0, 0) : g.pop_off(-cx(i), -cy(i), -cz(i)));
      if (kChecked && !in_bounds(w.fault, (src - f) + slot * kTile, pairs, kFaultPopLoad))
        src = f - slot * kTile;
      cp_async(&buf[b][i][tid], src + slot * kTile);
    }
  };
  auto decode = [&](int b, int own, float (&v1)[kQ], float (&v2)[kQ]) {
    const float2 own_prev =
        storage_local(ST)
            ? __ldg(&w.rho_enc[(kChecked && !in_bounds(w.fault, own, nodes, kFaultRhoLoad)) ? 0 : own])
            : make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float2 v = C::dec(buf[b][i][tid], dec_ref<ST>(p, own_prev, i));
      v1[i] = v.x;
      v2[i] = v.y;
    }
  };
  const int grp = (int)(k / (unsigned)a.tp), T = (int)(k % (unsigned)a.tp);
  const int tx = T % p.ntx, ty = T / p.ntx;
  const int x = tx * kTile + threadIdx.x, y = ty * BY + threadIdx.y;
  const bool active = x < p.nx && y < p.ny;
  const int q = grp - a.lag;                     // plane collided, if >= 0
  const int zd = grp == 0 ? p.nz - 1 : grp - 1;  // plane summed, if grp < nz
  const bool has_c = q >= 0, has_d = grp < p.nz;
  const int xlo = tx * kTile, xhi = min(xlo + kTile, p.nx) - 1;
  const int ylo = ty * BY, yhi = min(ylo + BY, p.ny) - 1;
  // one commit group per plane: the collision's first
  if (has_c && active) copy(x, y, q, 0);
  cp_async_commit();
  if (has_d && active) copy(x, y, zd, 1);
  cp_async_commit();
  // every warp waits for the 27 tiles' densities itself
  if (has_c && threadIdx.x < 27) {
    const int l = threadIdx.x;
    const int dx = l % 3 - 1, dy = (l / 3) % 3 - 1, dz = l / 9 - 1;
    const int zz = (q + dz + p.nz) % p.nz, yy = (ty + dy + nty) % nty,
              xx = (tx + dx + p.ntx) % p.ntx;
    long long fi = (long long)zz * a.tp + (long long)yy * p.ntx + xx;
    if (kChecked && !in_bounds(w.fault, fi, nflags, kFaultFlag)) fi = 0;
    // after one wait of this launch has run out the others give up at once
    unsigned n = 0;
    while (ld_relaxed(&flag[fi]) != epoch) {
      if (++n == a.spin_limit) {
        wave_fault(w, epoch);
        break;
      }
      if ((n & 255u) == 0 && *(volatile unsigned *)&ctl[3] == epoch) break;
      __nanosleep(64);
    }
  }
  __syncwarp();  // the densities this warp's collisions read are published
  if (has_c && active) {
    cp_async_wait<1>();
    const Geo g = make_geo(p, x, y, q);
    float f1[kQ], f2[kQ];
    decode(0, g.node(0, 0, 0), f1, f2);
    reservoir_state(p, box_in_reservoir(p, xlo, xhi, ylo, yhi, q, q), x, y, q, f1, f2);
    collide_loaded<PARITY, ST, PC, WaveRho>(p, w, g, WaveRho{global_rho(p, w, g)}, f1, f2);
  }
  cp_async_wait<0>();
  if (has_d && active) {
    const long long own = ((long long)(zd * p.ny + y) * p.ntx + tx) * kTile + threadIdx.x;
    float v1[kQ], v2[kQ];
    decode(1, (int)own, v1, v2);
    reservoir_state(p, box_in_reservoir(p, xlo, xhi, ylo, yhi, zd, zd), x, y, zd, v1, v2);
    if (in_bounds(w.fault, own, nodes, kFaultRhoStore))
      w.rho[own] = make_float2(sum19(v1), sum19(v2));
  }
  __syncthreads();  // the tile's densities are stored, the buffers free
  if (has_d && tid == 0) {
    long long fi = (long long)zd * a.tp + T;
    if (fi != hold && (!kChecked || in_bounds(w.fault, fi, nflags, kFaultFlag)))
      st_release(&flag[fi], epoch);
  }
}

// The last block out resets the ticket and done counter (in ctl) and
// advances the epoch of each of the launch's n lattices (ctls[l][2]) for
// the next launch.
__device__ __forceinline__ void wave_exit(unsigned *ctl, unsigned *const *ctls, int n) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    if (atomicAdd(&ctl[1], 1u) == gridDim.x - 1) {
      volatile unsigned *vc = ctl;
      vc[0] = 0u;
      vc[1] = 0u;
      for (int l = 0; l < n; ++l) {
        volatile unsigned *e = ctls[l];
        e[2] = e[2] + 1u;
      }
      __threadfence();
    }
  }
}

template <int PARITY, int ST, bool PC, int CFG>
__global__ void __launch_bounds__(WaveShape<ST, CFG>::threads, WaveShape<ST, CFG>::minb)
    k_wave(StepParams p, Workspace w, WaveArgs a) {
  using T2 = typename Codec2<ST>::T2;
  constexpr int BY = WaveShape<ST, CFG>::c.by, NT = kTile * BY;
  extern __shared__ __align__(16) unsigned char wave_smem[];
  T2(*buf)[kQ][NT] = reinterpret_cast<T2(*)[kQ][NT]>(wave_smem);  // [0] collision, [1] density
  __shared__ unsigned s_ticket[2], s_epoch;
  const int tid = threadIdx.y * kTile + threadIdx.x;
  unsigned *ctl = w.wave;
  if (tid == 0) {
    s_epoch = *(volatile unsigned *)&ctl[2] + 1u;
    s_ticket[0] = atomicAdd(&ctl[0], 1u);
  }
  __syncthreads();
  const unsigned epoch = s_epoch;
  unsigned k = s_ticket[0];
  int it = 0;
  while (k < a.items) {
    it ^= 1;
    if (tid == 0) s_ticket[it] = atomicAdd(&ctl[0], 1u);  // next item, read at the end
    wave_tile_item<PARITY, ST, PC, BY>(p, w, k, a, a.hold, buf, epoch);
    k = s_ticket[it];
  }
  unsigned *ctls[1] = {ctl};
  wave_exit(ctl, ctls, 1);
}

// ---- single-pass step: density and fused pass in one sweep ----
//
// The two-pass step reads every population twice (160 B/node for the
// density pass).  A single sweep must know the densities of a node's
// neighbours before it collides the node, and a block cannot recompute a
// neighbour's density from that neighbour's populations if another block may
// already have updated them in place.  So the lattice is cut into boxes of
// full x-rows: rows [y0, y0 + kSpBY) and nzc runs of planes along z (run c
// covers [c nz / nzc, (c + 1) nz / nzc), so runs differ by one plane at
// most and the grid is nyb x nzc boxes, a number the host can fit to the
// SM count).  The last row
// and the last plane of every box are seams.  One launch (k_sp_bulk) marches
// each box along z; per plane it computes the densities of the next plane --
// its own rows plus the seam row of the box below -- into a shared-memory
// ring of four planes, and collides the plane's bulk rows with the force
// stencil read from the ring.  Every density a box needs belongs to one of
// its own nodes (computed before that node is updated) or to a seam of
// another box (not updated by this launch).  Each box writes the densities of
// its own nodes to the density array; a second launch (k_sp_seams) then
// updates the seam rows and planes with the two-pass code, reading the
// completed array.  In-place AA streaming keeps every write of a node inside
// that node's own (slot, node) set, so no update disturbs another node's
// reads.  Results are bit-identical to the two-pass step (same densities,
// same arithmetic).
constexpr int kSpBY = 8;            // rows per box, the last one a seam
constexpr int kSpMaxThreads = 256;  // one thread per x: nx <= 256
constexpr int kSpRingPlanes = 4;

// First plane of run c of nzc runs along nz planes.
__host__ __device__ __forceinline__ int sp_run_start(int c, int nz, int nzc) {
  return (int)(((long long)c * nz) / nzc);
}

__host__ __device__ constexpr size_t sp_ring_bytes(int ncol) {
  return sizeof(float2) * kSpRingPlanes * (kSpBY + 1) * (size_t)ncol;
}

// Densities of x +- 1, y +- 1, z +- 1 from the ring.
struct RingRho {
  const float2 *row[3];  // ring row of the node's y in planes z - 1, z, z + 1
  int stride;            // one ring row (columns)
  int xm, xc, xp;        // columns of x - 1, x, x + 1 (periodic)
  const float2 *base;    // the ring and its length (bounds-checked builds)
  long long size;
  unsigned *fault;
  const GlobalRho *glob; // adhesion sources come from global memory
  __device__ __forceinline__ float2 at(int dx, int dy, int dz) const {
    const float2 *q = row[dz + 1] + dy * stride + (dx < 0 ? xm : (dx > 0 ? xp : xc));
    if (kChecked && !in_bounds(fault, q - base, size, kFaultShared)) q = base;
    return *q;
  }
  __device__ __forceinline__ float2 late(int dx, int dy, int dz) const {
    return at(dx, dy, dz);
  }
  __device__ __forceinline__ float a1(int dx, int dy, int dz) const {
    return glob->a1(dx, dy, dz);
  }
  __device__ __forceinline__ float a2(int dx, int dy, int dz) const {
    return glob->a2(dx, dy, dz);
  }
};

// Density pair of node (x, y, z) at the current step.
template <int PARITY, int ST>
__device__ __forceinline__ float2 node_density(const StepParams &p, const Workspace &w,
                                               const Geo &g, int x, int y, int z) {
  float v1[kQ], v2[kQ];
  load_pops<PARITY, ST>(p, w, g, v1, v2);
  reservoir_state(p, p.res.any != 0, x, y, z, v1, v2);
  return make_float2(sum19(v1), sum19(v2));
}

template <int PARITY, int ST, bool PC>
__global__ void __launch_bounds__(kSpMaxThreads, 2)
    k_sp_bulk(StepParams p, Workspace w, int nzc) {
  extern __shared__ float2 ring[];  // [kSpRingPlanes][kSpBY + 1][ncol]
  const int ncol = blockDim.x;
  const int x = threadIdx.x;
  const bool active = x < p.nx;
  const int y0 = blockIdx.x * kSpBY, yend = min(y0 + kSpBY, p.ny);
  const int nr = yend - y0;  // own rows; ring row r <-> y0 - 1 + r
  const int z0 = sp_run_start(blockIdx.y, p.nz, nzc);
  const int zend = sp_run_start(blockIdx.y + 1, p.nz, nzc);
  const int plane_stride = (kSpBY + 1) * ncol;

  // densities of relative plane k (z = z0 - 1 + k) into ring slot k % 4;
  // own nodes (rows 1..nr, planes z0..zend-1) also go to the density array
  auto rho_plane = [&](int k) {
    int z = z0 - 1 + k;
    const bool own_plane = k >= 1;
    if (z < 0) z += p.nz;
    float2 *dst = ring + (k & 3) * plane_stride;
    if (!active) return;
#pragma unroll 2
    for (int r = 0; r <= nr; ++r) {
      int y = y0 - 1 + r;
      if (y < 0) y += p.ny;
      const Geo g = make_geo(p, x, y, z);
      const float2 rho = node_density<PARITY, ST>(p, w, g, x, y, z);
      if (in_bounds(w.fault, (dst - ring) + r * ncol + x,
                    (long long)kSpRingPlanes * plane_stride, kFaultShared))
        dst[r * ncol + x] = rho;
      const int own = g.node(0, 0, 0);
      if (own_plane && r >= 1 && in_bounds(w.fault, own, p.ntiles * kTile, kFaultRhoStore))
        w.rho[own] = rho;
    }
  };

  rho_plane(0);
  rho_plane(1);
  const int xm = x == 0 ? p.nx - 1 : x - 1;
  const int xp = x == p.nx - 1 ? 0 : x + 1;
  for (int j = 0; j + 1 < zend - z0; ++j) {
    rho_plane(j + 2);
    __syncthreads();
    if (!active) continue;
    const int z = z0 + j;
    for (int r = 1; r < nr; ++r) {
      const int y = y0 - 1 + r;
      const Geo g = make_geo(p, x, y, z);
      RingRho rr;
      rr.row[0] = ring + (j & 3) * plane_stride + r * ncol;
      rr.row[1] = ring + ((j + 1) & 3) * plane_stride + r * ncol;
      rr.row[2] = ring + ((j + 2) & 3) * plane_stride + r * ncol;
      rr.stride = ncol;
      rr.xm = xm;
      rr.xc = x;
      rr.xp = xp;
      rr.base = ring;
      rr.size = (long long)kSpRingPlanes * plane_stride;
      rr.fault = w.fault;
      const GlobalRho glob = global_rho(p, w, g);
      rr.glob = &glob;
      collide_node<PARITY, ST, PC>(p, w, g, rr, p.res.any != 0, x, y, z);
    }
  }
}

// Seam rows of every box (all planes), then seam planes of every box (the
// rows that are not seam rows): the two-pass fused update with the density
// array the bulk launch completed.  Blocks of 32 x 4 threads.
template <int PARITY, int ST, bool PC>
__global__ void __launch_bounds__(kTile * 4, 4)
    k_sp_seams(StepParams p, Workspace w, int nzc, int part) {
  const int x = blockIdx.x * kTile + threadIdx.x;
  int y, z;
  if (part == 0) {
    y = min(blockIdx.y * kSpBY + kSpBY - 1, p.ny - 1);
    z = blockIdx.z * 4 + threadIdx.y;
    if (z >= p.nz) return;
  } else {
    y = blockIdx.y * 4 + threadIdx.y;
    z = sp_run_start(blockIdx.z + 1, p.nz, nzc) - 1;
    if (y >= p.ny) return;
    const int yseam = min((y / kSpBY) * kSpBY + kSpBY - 1, p.ny - 1);
    if (y == yseam) return;
  }
  if (x >= p.nx) return;
  collide_body<PARITY, ST, PC>(p, w, p.res.any != 0, x, y, z);
}

// ---- batched kernels: several lattices per launch ----

__device__ __forceinline__ int batch_item_of_block(const BatchArgs &a) {
  int lo = 0, hi = a.n - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.prefix[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Node coordinates of this thread inside its item; false for padding.
__device__ __forceinline__ bool batch_coords(const BatchArgs &a, int &r, int &x,
                                             int &y, int &z, bool &maybe_res) {
  r = batch_item_of_block(a);
  const BatchItem &it = a.item[r];
  const int lb = blockIdx.x - a.prefix[r];
  const int bx = lb % it.gx, rest = lb / it.gx;
  const int by = rest % it.gy, bz = rest / it.gy;
  x = bx * kTile + threadIdx.x;
  y = by * kBatchBY + threadIdx.y;
  z = bz;
  maybe_res = box_in_reservoir(it.p, bx * kTile, min(bx * kTile + kTile, it.p.nx) - 1,
                               by * kBatchBY, min(by * kBatchBY + kBatchBY, it.p.ny) - 1,
                               z, z);
  return x < it.p.nx && y < it.p.ny;
}

template <int ST>
__global__ void __launch_bounds__(kTile * kBatchBY)
    k_batch_density(const __grid_constant__ BatchArgs a) {
  int r, x, y, z;
  bool maybe_res;
  if (!batch_coords(a, r, x, y, z, maybe_res)) return;
  const BatchItem &it = a.item[r];
  const Geo g = make_geo(it.p, x, y, z);
  float v1[kQ], v2[kQ];
  if (it.parity == 0)
    load_pops<0, ST>(it.p, it.w, g, v1, v2);
  else
    load_pops<1, ST>(it.p, it.w, g, v1, v2);
  reservoir_state(it.p, maybe_res, x, y, z, v1, v2);
  const int own = g.node(0, 0, 0);
  if (in_bounds(it.w.fault, own, it.p.ntiles * kTile, kFaultRhoStore))
    it.w.rho[own] = make_float2(sum19(v1), sum19(v2));
}

// All items of one launch have per-component fractions (PC) or none do.
template <int ST, bool PC>
__global__ void __launch_bounds__(kTile * kBatchBY, CollideShape<1, ST, 0>::s.minb)
    k_batch_collide(const __grid_constant__ BatchArgs a) {
  int r, x, y, z;
  bool maybe_res;
  if (!batch_coords(a, r, x, y, z, maybe_res)) return;
  const BatchItem &it = a.item[r];
  if (it.parity == 0)
    collide_body<0, ST, PC>(it.p, it.w, maybe_res, x, y, z);
  else
    collide_body<1, ST, PC>(it.p, it.w, maybe_res, x, y, z);
}

// Blocks per SM the batched prefetching pass is compiled for: those of the
// single-lattice kernel, except the local storages' odd step in shape 9,
// whose budget (6 blocks, up to 170 registers) lets the lattice lookup take
// it to 137 registers and 7 resident blocks; held to 8 blocks (128
// registers) it needs no spill.
template <int PARITY, int ST, int CFG>
__host__ __device__ constexpr int batch_pipe_minb() {
  return (storage_local(ST) && PARITY == 1 && CFG == 9) ? 8
                                                        : CollideShape<PARITY, ST, CFG>::s.minb;
}

// The prefetching fused pass over a batch of lattices at one AA parity:
// item r's blocks (prefix[r] .. prefix[r + 1]) tile its lattice as
// k_collide_pipe's grid does for shape CFG (gx x-tiles, gy row groups, runs
// of zc planes), and each block runs that kernel's body on its lattice.
template <int PARITY, int ST, bool PC, int CFG>
__global__ void __launch_bounds__(CollideShape<PARITY, ST, CFG>::threads,
                                  batch_pipe_minb<PARITY, ST, CFG>())
    k_batch_collide_pipe(const __grid_constant__ BatchArgs a) {
  const int r = batch_item_of_block(a);
  const BatchItem &it = a.item[r];
  const int lb = blockIdx.x - a.prefix[r];
  const int rest = lb / it.gx;
  pipe_block<PARITY, ST, PC, CFG>(it.p, it.w, lb % it.gx, rest % it.gy, rest / it.gy);
}

}  // namespace
}  // namespace hmcsc
