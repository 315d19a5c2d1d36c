/*
 * hmcsc_oracle.c -- plain FP64 CPU oracle of the homogenized multi-component
 * Shan-Chen (HMCSC) lattice Boltzmann step, D3Q19.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the method computes; the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark use it to check the CUDA path.  The
 * product path never links, loads or calls it, and it shares no code, header,
 * table or helper with the CUDA library.
 *
 * Paper: "Homogenized lattice Boltzmann model for simulating multi-phase
 * flows in heterogeneous porous media" (arXiv 2206.11524).
 *
 * The step follows the paper's equations in the paper's order:
 *   1. moments rho_sigma = sum_i f_i,sigma, j_sigma = sum_i f_i,sigma c_i
 *      (Eqs. A.4, A.5, Appendix A.2);
 *   2. fluid-fluid force F_inter (Eq. 3), fluid-solid force F_ads (Eq. 4),
 *      body force F_ext,sigma (Eq. 5), F_tot = their sum (Sec. 2);
 *   3. equilibrium velocity u^eq_sigma with the Shan-Chen force shift (Eq. 6);
 *   4. Maxwell-Boltzmann equilibrium f^eq (Eq. A.3);
 *   5. gray collision with partial bounce-back of the pre-collision
 *      populations (Eq. 1, Eq. A.2);
 *   6. streaming to x + c_i (left-hand side of Eq. 1);
 *   7. density reservoirs: the prescribed layers are reset to equilibrium at
 *      the prescribed densities and zero velocity (Sec. 4), or at a
 *      prescribed velocity (velocity boundary cells, Sec. 3.1).
 *
 * Storage: two population buffers (the step writes a fresh buffer; pull and
 * push are not mixed), layout f[sigma][i][n], n = x + nx*(y + ny*z).
 * The lattice is periodic on every axis for streaming and for the force
 * stencils; walls are n_s = 1 cells and open faces are density reservoirs.
 *
 * The bounce-back fraction is a field per component, n_s,sigma(x) (Eq. 1);
 * it enters the collision of its own component, the adhesion indicator
 * s = n_s,sigma of Eq. 4 and the fluid fraction of Eq. 7.  Arrays hold it as
 * ns[sigma][n]; n_s,1 = n_s,2 is the common case (Table 1).
 *
 * Readings of the paper taken here where it is silent:
 *   - the pseudopotential is the density itself (Eq. 3 uses rho);
 *   - G_ads is a per-node field, taken at the neighbour inside the sum of
 *     Eq. 4, with G_ads,1 = -G_ads,2 (Table 1);
 *   - every cell, n_s = 1 included, carries both components (Sec. 2);
 *   - reservoir corners: faces are applied in the order -x,+x,-y,+y,-z,+z,
 *     a later face overwriting an earlier one;
 *   - the saturation S_1 (Eq. 19) weights a cell by the fluid fraction of
 *     fluid 1, 1 - n_s,1.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp].
 */
#include <math.h>
#include <stddef.h>
#include <string.h>

#define Q 19

/* D3Q19 velocity set in the paper's ordering (Eq. A.8): c_{i+9} = -c_i for
 * i = 1..9.  Weights 1/3, 1/18 (|c| = 1), 1/36 (|c| = sqrt 2). */
static const int CX[Q] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0};
static const int CY[Q] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1, 0, 1, 0, 1, -1, 0, 0, 1, 1};
static const int CZ[Q] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1};

static double weight_of(int i) {
  int n2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
  if (n2 == 0) return 1.0 / 3.0;
  if (n2 == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* w_i, tabulated once from weight_of(). */
static double W[Q];
static int W_ready = 0;
static void init_weights(void) {
  if (W_ready) return;
  for (int i = 0; i < Q; ++i) W[i] = weight_of(i);
  W_ready = 1;
}
static double weight(int i) { return W[i]; }

/* Opposite direction i-bar (Appendix A: c_ibar = -c_i). Found by search so
 * that it does not depend on the i <-> i+9 pattern being typed correctly. */
static int opposite(int i) {
  for (int k = 0; k < Q; ++k)
    if (CX[k] == -CX[i] && CY[k] == -CY[i] && CZ[k] == -CZ[i]) return k;
  return -1;
}

static const double CS2 = 1.0 / 3.0; /* lattice speed of sound squared */

typedef struct {
  int nx, ny, nz;
  double tau[2];     /* relaxation times tau_sigma                (Eq. 1)  */
  double G;          /* G_inter,12 = G_inter,21                   (Eq. 3)  */
  double Fext[3];    /* body force on the mixture                 (Eq. 5)  */
  int res_layers[6]; /* reservoir thickness per face, 0 = none (Sec. 4)    */
  double res_rho[6][2]; /* prescribed densities per face and component     */
  double res_u[6][3];   /* prescribed velocity per face (0: density
                           reservoir; nonzero: the velocity boundary cells of
                           the Couette flow, Sec. 3.1)                      */
} orc_params;

/* Periodic wrap of one coordinate into [0, n). */
static int wrap(int x, int n) {
  while (x < 0) x += n;
  while (x >= n) x -= n;
  return x;
}

static size_t node(const orc_params *p, int x, int y, int z) {
  x = wrap(x, p->nx);
  y = wrap(y, p->ny);
  z = wrap(z, p->nz);
  return (size_t)x + (size_t)p->nx * ((size_t)y + (size_t)p->ny * (size_t)z);
}

static size_t n_nodes(const orc_params *p) {
  return (size_t)p->nx * (size_t)p->ny * (size_t)p->nz;
}

/* Address of f_i,sigma at node n in f[sigma][i][n]. */
static size_t fidx(const orc_params *p, int s, int i, size_t n) {
  return ((size_t)s * Q + (size_t)i) * n_nodes(p) + n;
}

/* Which reservoir (last face in -x,+x,-y,+y,-z,+z order wins) holds node
 * (x,y,z); -1 if none.  Sec. 4: "reservoirs had a thickness of four layers". */
static int reservoir_face(const orc_params *p, int x, int y, int z) {
  int face = -1;
  if (p->res_layers[0] > 0 && x < p->res_layers[0]) face = 0;
  if (p->res_layers[1] > 0 && x >= p->nx - p->res_layers[1]) face = 1;
  if (p->res_layers[2] > 0 && y < p->res_layers[2]) face = 2;
  if (p->res_layers[3] > 0 && y >= p->ny - p->res_layers[3]) face = 3;
  if (p->res_layers[4] > 0 && z < p->res_layers[4]) face = 4;
  if (p->res_layers[5] > 0 && z >= p->nz - p->res_layers[5]) face = 5;
  return face;
}

/* G_ads,sigma at node n: G_ads,2 is the stored field, G_ads,1 = -G_ads,2
 * (Table 1). */
static double gads_of(const double *gads2, int s, size_t n) {
  return s == 0 ? -gads2[n] : gads2[n];
}

/* ---- lattice tables, exported so tests can check them independently ---- */
void orc_lattice(int *c /*[19][3]*/, double *w /*[19]*/, int *opp /*[19]*/) {
  init_weights();
  for (int i = 0; i < Q; ++i) {
    c[3 * i + 0] = CX[i];
    c[3 * i + 1] = CY[i];
    c[3 * i + 2] = CZ[i];
    w[i] = weight(i);
    opp[i] = opposite(i);
  }
}

/* Maxwell-Boltzmann equilibrium (Eq. A.3) for one direction. */
static double feq(int i, double rho, const double u[3]) {
  double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return weight(i) * rho *
         (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Exported for the tests: f^eq_i(rho, u) for all 19 directions. */
void orc_feq(double rho, const double *u, double *out /*[19]*/) {
  init_weights();
  for (int i = 0; i < Q; ++i) out[i] = feq(i, rho, u);
}

/* Initial state f_i,sigma = f^eq_i(rho_sigma, u = 0): the domain is
 * "initially filled with" given densities at rest (Secs. 3.3, 3.4, 4). */
void orc_init_equilibrium(const orc_params *p, const double *rho_a,
                          const double *rho_b, double *f) {
  init_weights();
  const size_t N = n_nodes(p);
  const double zero[3] = {0.0, 0.0, 0.0};
  for (size_t n = 0; n < N; ++n)
    for (int i = 0; i < Q; ++i) {
      f[fidx(p, 0, i, n)] = feq(i, rho_a[n], zero);
      f[fidx(p, 1, i, n)] = feq(i, rho_b[n], zero);
    }
}

/* Zeroth and first moments of component s at node n (Eqs. A.4, A.5; the
 * first moment is kept as the momentum density j = rho u). */
static void moments(const orc_params *p, const double *f, int s, size_t n,
                    double *rho, double j[3]) {
  *rho = 0.0;
  j[0] = j[1] = j[2] = 0.0;
  for (int i = 0; i < Q; ++i) {
    double fi = f[fidx(p, s, i, n)];
    *rho += fi;
    j[0] += fi * CX[i];
    j[1] += fi * CY[i];
    j[2] += fi * CZ[i];
  }
}

/* Total force on component s at node (x,y,z), from the densities of the whole
 * lattice at the same time (rho[2][N]):
 *   F_inter,s = -rho_s G sum_i w_i rho_sbar(x + c_i) c_i              (Eq. 3)
 *   F_ads,s   = -rho_s sum_i w_i G_ads,s(x + c_i) n_s,s(x + c_i) c_i  (Eq. 4)
 *   F_ext,s   = rho_s / rho * F_ext                                 (Eq. 5)
 */
static void total_force(const orc_params *p, const double *rho,
                        const double *ns, const double *gads2, int s, int x,
                        int y, int z, double F[3]) {
  const size_t N = n_nodes(p);
  const size_t n = node(p, x, y, z);
  const int sb = 1 - s;
  const double rho_s = rho[(size_t)s * N + n];
  const double rho_tot = rho[n] + rho[N + n];
  double S[3] = {0.0, 0.0, 0.0}; /* sum_i w_i rho_sbar(x+c_i) c_i      */
  double A[3] = {0.0, 0.0, 0.0}; /* sum_i w_i Gads(x+c_i) ns_s(x+c_i) c_i */
  for (int i = 0; i < Q; ++i) {
    size_t m = node(p, x + CX[i], y + CY[i], z + CZ[i]);
    double r = weight(i) * rho[(size_t)sb * N + m];
    double a = weight(i) * gads_of(gads2, s, m) * ns[(size_t)s * N + m];
    S[0] += r * CX[i];
    S[1] += r * CY[i];
    S[2] += r * CZ[i];
    A[0] += a * CX[i];
    A[1] += a * CY[i];
    A[2] += a * CZ[i];
  }
  for (int d = 0; d < 3; ++d) {
    double F_inter = -rho_s * p->G * S[d];
    double F_ads = -rho_s * A[d];
    double F_ext = rho_s / rho_tot * p->Fext[d];
    F[d] = F_inter + F_ads + F_ext;
  }
}

static void density_field(const orc_params *p, const double *f, double *rho) {
  const size_t N = n_nodes(p);
#pragma omp parallel for collapse(2) schedule(static)
  for (int s = 0; s < 2; ++s)
    for (size_t n = 0; n < N; ++n) {
      double r = 0.0;
      for (int i = 0; i < Q; ++i) r += f[fidx(p, s, i, n)];
      rho[(size_t)s * N + n] = r;
    }
}

/*
 * One time step t -> t+1.
 *   ns    [2][N]      bounce-back fraction n_s,sigma per component
 *   gads2 [N]         G_ads,2 per node
 *   f_in  [2][19][N]  state at t (read only)
 *   f_out [2][19][N]  state at t+1 (written)
 *   rho   [2][N]      scratch: densities at t
 *   post  [2][19][N]  scratch: post-collision populations
 */
void orc_step(const orc_params *p, const double *ns, const double *gads2,
              const double *f_in, double *f_out, double *rho, double *post) {
  init_weights();
  const size_t N = n_nodes(p);
  int opp[Q];
  for (int i = 0; i < Q; ++i) opp[i] = opposite(i);

  /* 1. densities of the whole lattice at time t (Eq. A.4): the forces of
   *    Eqs. 3-4 read them at the neighbours. */
  density_field(p, f_in, rho);

  /* 2-5. forces, equilibrium velocity, equilibrium, gray collision. */
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        const size_t n = node(p, x, y, z);
        double rho_s[2], j_s[2][3], F[2][3];
        for (int s = 0; s < 2; ++s) {
          moments(p, f_in, s, n, &rho_s[s], j_s[s]);
          total_force(p, rho, ns, gads2, s, x, y, z, F[s]);
        }
        /* common velocity: sum_s rho_s u_s / tau_s over sum_s rho_s / tau_s
         * (first term of Eq. 6) */
        double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
        for (int s = 0; s < 2; ++s) {
          for (int d = 0; d < 3; ++d) num[d] += j_s[s][d] / p->tau[s];
          den += rho_s[s] / p->tau[s];
        }
        for (int s = 0; s < 2; ++s) {
          double ueq[3];
          for (int d = 0; d < 3; ++d)
            ueq[d] = num[d] / den + p->tau[s] * F[s][d] / rho_s[s]; /* Eq. 6 */
          const double nsx = ns[(size_t)s * N + n];
          for (int i = 0; i < Q; ++i) {
            const double fi = f_in[fidx(p, s, i, n)];
            const double fbar = f_in[fidx(p, s, opp[i], n)]; /* pre-collision */
            const double fe = feq(i, rho_s[s], ueq);
            /* Eq. 1: fluid part relaxes, bounce-back part reflects. */
            post[fidx(p, s, i, n)] = (1.0 - nsx) * fi -
                                     (1.0 - nsx) / p->tau[s] * (fi - fe) +
                                     nsx * fbar;
          }
        }
      }

  /* 6. streaming: f_i(x + c_i, t + 1) = post_i(x). */
#pragma omp parallel for collapse(3) schedule(static)
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < Q; ++i)
      for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
          for (int x = 0; x < p->nx; ++x) {
            size_t from = node(p, x, y, z);
            size_t to = node(p, x + CX[i], y + CY[i], z + CZ[i]);
            f_out[fidx(p, s, i, to)] = post[fidx(p, s, i, from)];
          }

  /* 7. reservoirs: prescribed densities at rest (Sec. 4) or at the
   *    prescribed velocity of a velocity boundary (Sec. 3.1). */
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        int face = reservoir_face(p, x, y, z);
        if (face < 0) continue;
        size_t n = node(p, x, y, z);
        for (int s = 0; s < 2; ++s)
          for (int i = 0; i < Q; ++i)
            f_out[fidx(p, s, i, n)] = feq(i, p->res_rho[face][s], p->res_u[face]);
      }
}

/* Run n steps in place on f (two-buffer ping-pong through `tmp`). */
void orc_run(const orc_params *p, const double *ns, const double *gads2,
             double *f, double *tmp, double *rho, double *post, int steps) {
  const size_t total = 2 * (size_t)Q * n_nodes(p);
  for (int t = 0; t < steps; ++t) {
    orc_step(p, ns, gads2, f, tmp, rho, post);
    memcpy(f, tmp, total * sizeof(double));
  }
}

/*
 * Macroscopic fields of the state f at time t:
 *   rho_sigma                                                  (Eq. A.4)
 *   u_macro = 1/rho sum_s (1 - n_s,s)(j_s + F_tot,s / 2)       (Eq. 7)
 *   p = c_s^2 [rho + G rho_1 rho_2]                            (Eq. A.6)
 *   F_tot,sigma                                                (Eqs. 3-5)
 * Any output pointer may be NULL.  rho_scratch: [2][N].
 */
void orc_fields(const orc_params *p, const double *ns, const double *gads2,
                const double *f, double *rho_scratch, double *rho_a,
                double *rho_b, double *u /*[3][N]*/, double *pres,
                double *ftot /*[2][3][N]*/) {
  init_weights();
  const size_t N = n_nodes(p);
  density_field(p, f, rho_scratch);
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        const size_t n = node(p, x, y, z);
        double rho_s[2], j_s[2][3], F[2][3];
        for (int s = 0; s < 2; ++s) {
          moments(p, f, s, n, &rho_s[s], j_s[s]);
          total_force(p, rho_scratch, ns, gads2, s, x, y, z, F[s]);
        }
        const double rho = rho_s[0] + rho_s[1];
        if (rho_a) rho_a[n] = rho_s[0];
        if (rho_b) rho_b[n] = rho_s[1];
        if (u)
          for (int d = 0; d < 3; ++d) {
            double m = 0.0;
            for (int s = 0; s < 2; ++s)
              m += (1.0 - ns[(size_t)s * N + n]) * (j_s[s][d] + F[s][d] / 2.0);
            u[(size_t)d * N + n] = m / rho;
          }
        if (pres) pres[n] = CS2 * (rho + p->G * rho_s[0] * rho_s[1]);
        if (ftot)
          for (int s = 0; s < 2; ++s)
            for (int d = 0; d < 3; ++d)
              ftot[((size_t)s * 3 + d) * N + n] = F[s][d];
      }
}

/*
 * Scalar observables of the state f (Sec. 4):
 *   out[0], out[1]  mass of component 1 and 2: sum_x rho_sigma
 *   out[2]          saturation S_1 (Eq. 19): cells outside the reservoirs,
 *                   each weighted by its fluid-1 fraction (1 - n_s,1), counted
 *                   when rho_1 >= 0.5
 *   out[3 + k]      mean pressure (Eq. A.6) over the layers of reservoir
 *                   face k (k = 0..5: -x,+x,-y,+y,-z,+z), NaN if none;
 *                   Eq. 18's Delta p is the inlet mean minus the outlet mean.
 * rho_scratch: [2][N].
 */
/* Observables of given density fields rho[2][N] (Sec. 4): masses, S_1 of
 * Eq. 19, mean Eq. A.6 pressure of each reservoir face. */
void orc_observables_rho(const orc_params *p, const double *ns, const double *rho_scratch,
                         double *out /*[9]*/) {
  const size_t N = n_nodes(p);
  double mass[2] = {0.0, 0.0}, sat_num = 0.0, sat_den = 0.0;
  double psum[6] = {0, 0, 0, 0, 0, 0};
  double pcnt[6] = {0, 0, 0, 0, 0, 0};
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        size_t n = node(p, x, y, z);
        double r1 = rho_scratch[n], r2 = rho_scratch[N + n];
        mass[0] += r1;
        mass[1] += r2;
        /* a corner node counts toward every face whose layers contain it */
        const int in_face[6] = {
            p->res_layers[0] > 0 && x < p->res_layers[0],
            p->res_layers[1] > 0 && x >= p->nx - p->res_layers[1],
            p->res_layers[2] > 0 && y < p->res_layers[2],
            p->res_layers[3] > 0 && y >= p->ny - p->res_layers[3],
            p->res_layers[4] > 0 && z < p->res_layers[4],
            p->res_layers[5] > 0 && z >= p->nz - p->res_layers[5]};
        int in_any = 0;
        double pr = CS2 * (r1 + r2 + p->G * r1 * r2);
        for (int k = 0; k < 6; ++k)
          if (in_face[k]) {
            in_any = 1;
            psum[k] += pr;
            pcnt[k] += 1.0;
          }
        if (!in_any) {
          double wgt = 1.0 - ns[n];
          sat_den += wgt;
          if (r1 >= 0.5) sat_num += wgt;
        }
      }
  out[0] = mass[0];
  out[1] = mass[1];
  out[2] = sat_den > 0.0 ? sat_num / sat_den : NAN;
  for (int k = 0; k < 6; ++k) out[3 + k] = pcnt[k] > 0 ? psum[k] / pcnt[k] : NAN;
}

/* Observables of the current state: the densities of its populations, then
 * orc_observables_rho. */
void orc_observables(const orc_params *p, const double *ns, const double *f,
                     double *rho_scratch, double *out /*[9]*/) {
  init_weights();
  density_field(p, f, rho_scratch);
  orc_observables_rho(p, ns, rho_scratch, out);
}
