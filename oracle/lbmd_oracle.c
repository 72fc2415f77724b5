/*
 * lbmd_oracle.c -- FP64 CPU oracle of the coupled lattice-Boltzmann / polymer
 * molecular-dynamics step of Fyta, Melchionna, Kaxiras and Succi,
 * "Coupling Lattice Boltzmann with Atomistic Dynamics for the multiscale
 * simulation of nano-biological flows" (arXiv:0710.1272), Sec. II and Sec. III.
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant generator with the CUDA library and it
 * includes nothing from it.
 *
 * Everything is double precision.  The LB update is written in the textbook
 * "collide, then push" form of Eq. 5; the MD substep follows the Sec. II
 * description (Eqs. 1-4, SHAKE/RATTLE) with the readings listed next to each
 * function.  The per-LB-step order is the four-stage scheme of Sec. II:
 * interpolate u to the beads, run M MD substeps with u frozen, extrapolate the
 * bead forces to the grid, advance the populations.
 *
 * Readings where the paper is silent:
 *  - D3Q19 weights 1/3, 1/18, 1/36 and c_s^2 = 1/3 (Sec. II cites the standard
 *    19-speed lattice without printing them).
 *  - The fluid receives the reaction -(F_drag + F_r) of the bead forces in
 *    Eq. 10, so that fluid + bead momentum is conserved.
 *  - u is interpolated once per LB step at the start-of-step positions; the
 *    impulse J_i = sum_k dt_MD (F_drag + F_r) of the M substeps is spread with
 *    the same weights.
 *  - Trilinear weights (default) or nearest grid point (flag); solid corners
 *    are dropped and the fluid weights renormalised.
 *  - Random force variance from fluctuation-dissipation:
 *    <F_r F_r> = 2 m gamma kT / dt_MD per component.
 *  - LJ of Eq. 2 truncated at 2^(1/6) sigma (purely repulsive), over pairs that
 *    are not bonded; bead-wall force: the same potential between a bead and
 *    every solid node.
 *  - Explicit Euler-Langevin substep + SHAKE + RATTLE (the stochastic
 *    integrator of Sec. II is only cited).
 *  - Halfway bounce-back on solid nodes (the paper names no wall scheme).
 *
 * Parity status: every function here is pinned by a CPU test (closed forms,
 * conservation laws, finite differences, brute-force re-implementation on a
 * tiny box, published Philox test vectors).  The long-horizon trajectory of a
 * translocation event is chaotic and is compared statistically only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* D3Q19 velocity set; opposite directions are adjacent (1/2, 3/4, ...). */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},
    {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};

static double weight(int p) {
  if (p == 0) return 1.0 / 3.0;
  if (p <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}
static int opposite(int p) {
  if (p == 0) return 0;
  return (p % 2 == 1) ? p + 1 : p - 1;
}
static const double CS2 = 1.0 / 3.0; /* squared sound speed */

enum { ORC_PAPER = 0, ORC_GUO = 1 };
enum { ORC_TRILINEAR = 0, ORC_NGP = 1 };
enum {
  ORC_RUNNING = 0,
  ORC_TRANSLOCATED = 1,
  ORC_RETRACTED = 2,
  ORC_NAN = 3,
  ORC_SHAKE_FAIL = 4
};

typedef struct {
  int32_t nx, ny, nz;
  int32_t wall_x, wall_thickness;   /* wall_x < 0: no wall */
  int32_t pore_d, pore_y0, pore_z0; /* pore_d <= 0: closed; y0,z0 < 0: centred */
  int32_t y_walls;                  /* 1: solid rows y = 0 and y = ny-1 */
  int32_t forcing, coupling;
  int32_t n_beads, md_substeps;
  int32_t n_bonds;                  /* bonds given in the create call */
  int32_t shake_max_iter;
  int32_t hydrodynamics;            /* 0: solvent-free (u_i = 0, no LB) */
  double tau, rho0, g[3];
  double mass, gamma, kT, lj_sigma, lj_eps, kappa_phi, f_drive;
  double shake_tol;
  double kT_fluid;                  /* thermal source F_p of Eq. 5; 0: off */
  uint64_t seed;
} orc_params;

typedef struct {
  orc_params p;
  int64_t V;
  double *f, *fs;     /* pre-collision f(x,t) and post-collision f*(x,t) */
  double *rho, *u;    /* moments of f (u includes the Guo shift if set) */
  double *F;          /* bead force density on the grid, 3*V */
  uint8_t *solid;
  int32_t *bi, *bj;   /* bonds */
  double *b0;
  double *r, *v;      /* bead positions (unwrapped) and velocities, 3*N */
  double *ui, *J;     /* interpolated fluid velocity, impulse of last step */
  int64_t step;
  int32_t n_trans, max_trans, state;
  int64_t t_transloc;
  int32_t last_shake_sweeps, last_rattle_sweeps;
} orc_sim;

/* ------------------------------------------------------------------ */
/* Indexing helpers                                                    */
/* ------------------------------------------------------------------ */
static int wrapi(int a, int n) {
  int m = a % n;
  return m < 0 ? m + n : m;
}
static double wrapd(double a, double n) {
  double m = fmod(a, n);
  return m < 0 ? m + n : m;
}
static int64_t cell(const orc_sim *s, int x, int y, int z) {
  return ((int64_t)z * s->p.ny + y) * s->p.nx + x;
}

/* ------------------------------------------------------------------ */
/* Eq. 6: second-order equilibrium                                     */
/* ------------------------------------------------------------------ */
void orc_equilibrium(double rho, const double u[3], double feq[Q]) {
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int p = 0; p < Q; ++p) {
    double cu = CV[p][0] * u[0] + CV[p][1] * u[1] + CV[p][2] * u[2];
    /* uu:(cc - cs2 I) = (c.u)^2 - cs2 |u|^2 */
    feq[p] = weight(p) * rho *
             (1.0 + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
  }
}

/* Eqs. 7-8 (plus, for the Guo flag only, the half-force velocity shift). */
void orc_moments(const double f[Q], const double g[3], int forcing,
                 double *rho_out, double u_out[3]) {
  double rho = 0, m[3] = {0, 0, 0};
  for (int p = 0; p < Q; ++p) {
    rho += f[p];
    for (int a = 0; a < 3; ++a) m[a] += f[p] * CV[p][a];
  }
  for (int a = 0; a < 3; ++a) {
    if (forcing == ORC_GUO) m[a] += 0.5 * g[a];
    u_out[a] = m[a] / rho;
  }
  *rho_out = rho;
}

/* Eq. 5 collision at one node, Delta t = 1, omega = 1/tau, no thermal source.
 * Source S_p (Eq. 10 form, first order): (w_p / c_s^2) c_p . (g + Fb), where g
 * is the uniform body force density and Fb the bead reaction force density.
 * Guo flag: the body force enters through the velocity shift and the
 * second-order source (1 - 1/(2 tau)) w_p [(c - u)/cs2 + (c.u) c / cs2^2] . g;
 * the bead force keeps the first-order form. */
void orc_collide(const double f[Q], double tau, const double Fb[3],
                 const double g[3], int forcing, double out[Q]) {
  double rho, u[3], feq[Q];
  orc_moments(f, g, forcing, &rho, u);
  orc_equilibrium(rho, u, feq);
  for (int p = 0; p < Q; ++p) {
    double c[3] = {CV[p][0], CV[p][1], CV[p][2]};
    double src_b = weight(p) / CS2 * (c[0] * Fb[0] + c[1] * Fb[1] + c[2] * Fb[2]);
    double src_g;
    if (forcing == ORC_GUO) {
      double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
      double acc = 0;
      for (int a = 0; a < 3; ++a)
        acc += ((c[a] - u[a]) / CS2 + cu * c[a] / (CS2 * CS2)) * g[a];
      src_g = (1.0 - 0.5 / tau) * weight(p) * acc;
    } else {
      src_g = weight(p) / CS2 * (c[0] * g[0] + c[1] * g[1] + c[2] * g[2]);
    }
    out[p] = f[p] - (f[p] - feq[p]) / tau + src_g + src_b;
  }
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the  */
/* published round function: two 32x32->64 multiplies per round, the    */
/* key bumped by the Weyl constants between rounds.                     */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k[2] = {key_in[0], key_in[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += W0;
      k[1] += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c[0];
    uint64_t p1 = (uint64_t)M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
  memcpy(out, c, sizeof(c));
}

/* Uniform in (0,1) from the top 23 bits: ((x >> 9) + 1/2) 2^-23. */
static double uniform23(uint32_t x) {
  return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Three standard normal deviates for (bead, LB step, MD substep, stream) by
 * Box-Muller on the four uniforms of one Philox block.
 * key = (seed lo, seed hi); counter = (bead, step lo, step hi,
 * substep | stream << 8). */
void orc_gauss3(uint64_t seed, uint32_t bead, int64_t step, uint32_t substep,
                uint32_t stream, double xi[3]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {bead, (uint32_t)(uint64_t)step,
                     (uint32_t)((uint64_t)step >> 32),
                     (substep & 0xFFu) | (stream << 8)};
  uint32_t x[4];
  orc_philox4x32_10(ctr, key, x);
  double u1 = uniform23(x[0]), u2 = uniform23(x[1]);
  double u3 = uniform23(x[2]), u4 = uniform23(x[3]);
  double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
  const double two_pi = 6.283185307179586476925286766559;
  xi[0] = r1 * cos(two_pi * u2);
  xi[1] = r1 * sin(two_pi * u2);
  xi[2] = r2 * cos(two_pi * u4);
}

/* ------------------------------------------------------------------ */
/* Geometry (Sec. III): wall at x = wall_x, centred square pore of side  */
/* d, optional solid rows y = 0 and y = ny-1.                           */
/* ------------------------------------------------------------------ */
static void pore_origin(const orc_params *p, int *y0, int *z0) {
  *y0 = p->pore_y0 >= 0 ? p->pore_y0 : (p->ny - p->pore_d) / 2;
  *z0 = p->pore_z0 >= 0 ? p->pore_z0 : (p->nz - p->pore_d) / 2;
}

static void build_solid(orc_sim *s) {
  const orc_params *p = &s->p;
  int y0, z0;
  pore_origin(p, &y0, &z0);
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        int sol = 0;
        if (p->wall_x >= 0) {
          int in_wall = 0;
          for (int t = 0; t < p->wall_thickness; ++t)
            if (x == wrapi(p->wall_x + t, p->nx)) in_wall = 1;
          int in_pore = p->pore_d > 0 && y >= y0 && y < y0 + p->pore_d &&
                        z >= z0 && z < z0 + p->pore_d;
          if (in_wall && !in_pore) sol = 1;
        }
        if (p->y_walls && (y == 0 || y == p->ny - 1)) sol = 1;
        s->solid[cell(s, x, y, z)] = (uint8_t)sol;
      }
}

static int is_solid(const orc_sim *s, int x, int y, int z) {
  return s->solid[cell(s, wrapi(x, s->p.nx), wrapi(y, s->p.ny),
                       wrapi(z, s->p.nz))];
}

/* ------------------------------------------------------------------ */
/* Creation                                                            */
/* ------------------------------------------------------------------ */
void orc_destroy(orc_sim *s);

orc_sim *orc_create(const orc_params *pin, const int32_t *bond_i,
                    const int32_t *bond_j, const double *bond_len,
                    const double *init_pos, const double *init_vel,
                    const double *init_rho, const double *init_u) {
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  if (!s) return NULL;
  s->p = *pin;
  const orc_params *p = &s->p;
  s->V = (int64_t)p->nx * p->ny * p->nz;
  int64_t V = s->V;
  int N = p->n_beads;
  s->f = (double *)calloc((size_t)(Q * V), sizeof(double));
  s->fs = (double *)calloc((size_t)(Q * V), sizeof(double));
  s->rho = (double *)calloc((size_t)V, sizeof(double));
  s->u = (double *)calloc((size_t)(3 * V), sizeof(double));
  s->F = (double *)calloc((size_t)(3 * V), sizeof(double));
  s->solid = (uint8_t *)calloc((size_t)V, 1);
  int nb = p->n_bonds;
  s->bi = (int32_t *)calloc((size_t)(nb > 0 ? nb : 1), sizeof(int32_t));
  s->bj = (int32_t *)calloc((size_t)(nb > 0 ? nb : 1), sizeof(int32_t));
  s->b0 = (double *)calloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
  size_t nn = (size_t)(3 * (N > 0 ? N : 1));
  s->r = (double *)calloc(nn, sizeof(double));
  s->v = (double *)calloc(nn, sizeof(double));
  s->ui = (double *)calloc(nn, sizeof(double));
  s->J = (double *)calloc(nn, sizeof(double));
  if (!s->f || !s->fs || !s->rho || !s->u || !s->F || !s->solid || !s->bi ||
      !s->bj || !s->b0 || !s->r || !s->v || !s->ui || !s->J) {
    orc_destroy(s);
    return NULL;
  }
  for (int b = 0; b < nb; ++b) {
    s->bi[b] = bond_i[b];
    s->bj[b] = bond_j[b];
    s->b0[b] = bond_len[b];
  }
  if (N > 0) {
    memcpy(s->r, init_pos, sizeof(double) * 3 * N);
    if (init_vel) memcpy(s->v, init_vel, sizeof(double) * 3 * N);
  }
  build_solid(s);
  /* f(x, 0) = f_eq(rho(x), u(x)) at fluid nodes; zero at solid nodes. */
  for (int64_t c = 0; c < V; ++c) {
    if (s->solid[c]) continue;
    double rho = init_rho ? init_rho[c] : p->rho0;
    double u[3] = {0, 0, 0};
    if (init_u)
      for (int a = 0; a < 3; ++a) u[a] = init_u[a * V + c];
    double feq[Q];
    orc_equilibrium(rho, u, feq);
    for (int q = 0; q < Q; ++q) s->f[q * V + c] = feq[q];
  }
  s->t_transloc = -1;
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->f);
  free(s->fs);
  free(s->rho);
  free(s->u);
  free(s->F);
  free(s->solid);
  free(s->bi);
  free(s->bj);
  free(s->b0);
  free(s->r);
  free(s->v);
  free(s->ui);
  free(s->J);
  free(s);
}

/* ------------------------------------------------------------------ */
/* LB stages                                                           */
/* ------------------------------------------------------------------ */
static void compute_moments(orc_sim *s) {
  const int64_t V = s->V;
  const orc_params *p = &s->p;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < V; ++c) {
    if (s->solid[c]) {
      s->rho[c] = 0;
      s->u[c] = s->u[V + c] = s->u[2 * V + c] = 0;
      continue;
    }
    double f[Q], rho, u[3];
    for (int q = 0; q < Q; ++q) f[q] = s->f[q * V + c];
    orc_moments(f, p->g, p->forcing, &rho, u);
    s->rho[c] = rho;
    for (int a = 0; a < 3; ++a) s->u[a * V + c] = u[a];
  }
}

void orc_fluct_noise(uint64_t seed, uint32_t node, int64_t step, double rho, double tau,
                     double kT, double xi[Q]);

static void collide_all(orc_sim *s) {
  const int64_t V = s->V;
  const orc_params *p = &s->p;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < V; ++c) {
    if (s->solid[c]) continue;
    double f[Q], out[Q], Fb[3] = {s->F[c], s->F[V + c], s->F[2 * V + c]};
    for (int q = 0; q < Q; ++q) f[q] = s->f[q * V + c];
    orc_collide(f, p->tau, Fb, p->g, p->forcing, out);
    if (p->kT_fluid > 0) {
      double rho = 0.0, xi[Q];
      for (int q = 0; q < Q; ++q) rho += f[q];
      orc_fluct_noise(p->seed, (uint32_t)c, s->step, rho, p->tau, p->kT_fluid, xi);
      for (int q = 0; q < Q; ++q) out[q] += xi[q];
    }
    for (int q = 0; q < Q; ++q) s->fs[q * V + c] = out[q];
  }
}

/* Free streaming of Eq. 5 in push form: f_p(x + c_p, t+1) = f*_p(x, t); a
 * population whose destination is solid returns to x reversed (halfway
 * bounce-back). */
static void stream_all(orc_sim *s) {
  const orc_params *p = &s->p;
  const int64_t V = s->V;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        int64_t c = cell(s, x, y, z);
        if (s->solid[c]) continue;
        for (int q = 0; q < Q; ++q) {
          int xd = wrapi(x + CV[q][0], p->nx), yd = wrapi(y + CV[q][1], p->ny),
              zd = wrapi(z + CV[q][2], p->nz);
          int64_t d = cell(s, xd, yd, zd);
          if (!s->solid[d])
            s->f[q * V + d] = s->fs[q * V + c];
          else
            s->f[opposite(q) * V + c] = s->fs[q * V + c];
        }
      }
}

/* ------------------------------------------------------------------ */
/* Thermal source F_p of Eq. 5 (fluctuating LB, Adhikari et al. 2005; the */
/* mode form of Duenweg, Schiller and Ladd 2007): independent Gaussian    */
/* noise in every non-conserved mode of a weight-orthogonal basis, with   */
/* the variance that the fluctuation-dissipation theorem fixes for a      */
/* mode relaxing by the factor (1 - omega) per step.                      */
/* ------------------------------------------------------------------ */
/* Row k of the basis evaluated at c_p:
 * 0: 1; 1-3: c_x, c_y, c_z; 4: c^2 - 1; 5: 3c_x^2 - c^2; 6: c_y^2 - c_z^2;
 * 7-9: c_x c_y, c_y c_z, c_z c_x; 10-12: (3c^2 - 5) c_x, c_y, c_z;
 * 13: (c_y^2 - c_z^2) c_x; 14: (c_z^2 - c_x^2) c_y; 15: (c_x^2 - c_y^2) c_z;
 * 16: 3c^4 - 6c^2 + 1; 17: (2c^2 - 3)(3c_x^2 - c^2); 18: (2c^2 - 3)(c_y^2 - c_z^2). */
static double mode_row(int k, const int c[3]) {
  const double x = c[0], y = c[1], z = c[2], c2 = x * x + y * y + z * z;
  switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return z * x;
    case 10: return (3.0 * c2 - 5.0) * x;
    case 11: return (3.0 * c2 - 5.0) * y;
    case 12: return (3.0 * c2 - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    case 18: return (2.0 * c2 - 3.0) * (y * y - z * z);
  }
  return 0.0;
}

/* e[k][p] and the norms b_k = sum_p w_p e[k][p]^2. */
void orc_mode_basis(double e[Q][Q], double b[Q]) {
  for (int k = 0; k < Q; ++k) {
    b[k] = 0.0;
    for (int q = 0; q < Q; ++q) {
      e[k][q] = mode_row(k, CV[q]);
      b[k] += weight(q) * e[k][q] * e[k][q];
    }
  }
}

/* Fifteen standard normals for node `node` at LB step `step`: Box-Muller
 * on both pairs of uniforms of four Philox blocks, counter (node, step lo,
 * step hi, block | 2 << 8), key (seed lo, seed hi). */
static void fluct_normals(uint64_t seed, uint32_t node, int64_t step, double r[16]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two_pi = 6.283185307179586476925286766559;
  for (uint32_t j = 0; j < 4; ++j) {
    uint32_t ctr[4] = {node, (uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), j | (2u << 8)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    for (int h = 0; h < 2; ++h) {
      const double u1 = uniform23(x[2 * h]), u2 = uniform23(x[2 * h + 1]);
      const double rad = sqrt(-2.0 * log(u1));
      r[4 * j + 2 * h] = rad * cos(two_pi * u2);
      r[4 * j + 2 * h + 1] = rad * sin(two_pi * u2);
    }
  }
}

/* Thermal source of one node with density rho:
 *   xi_p = w_p sum_{k=4}^{18} e_kp / b_k * sqrt(mu b_k (1 - (1 - omega)^2)) r_k,
 *   mu = rho kT / c_s^2, omega = 1 / tau, r_k = normal number k - 4. */
void orc_fluct_noise(uint64_t seed, uint32_t node, int64_t step, double rho, double tau,
                     double kT, double xi[Q]) {
  double e[Q][Q], b[Q], r[16];
  orc_mode_basis(e, b);
  fluct_normals(seed, node, step, r);
  const double g1 = 1.0 - 1.0 / tau;
  const double mu = rho * kT / CS2;
  for (int q = 0; q < Q; ++q) xi[q] = 0.0;
  for (int k = 4; k < Q; ++k) {
    const double amp = sqrt(mu * b[k] * (1.0 - g1 * g1)) * r[k - 4] / b[k];
    for (int q = 0; q < Q; ++q) xi[q] += weight(q) * e[k][q] * amp;
  }
}

/* ------------------------------------------------------------------ */
/* Grid <-> bead transfer (Sec. II, Fig. 1)                            */
/* ------------------------------------------------------------------ */
/* Corner nodes and weights of one bead.  Returns the number of corners. */
static int transfer_weights(const orc_sim *s, const double r[3],
                            int64_t node[8], double w[8]) {
  const orc_params *p = &s->p;
  double L[3] = {p->nx, p->ny, p->nz};
  double rw[3];
  for (int a = 0; a < 3; ++a) rw[a] = wrapd(r[a], L[a]);
  if (p->coupling == ORC_NGP) {
    int x = wrapi((int)floor(rw[0] + 0.5), p->nx);
    int y = wrapi((int)floor(rw[1] + 0.5), p->ny);
    int z = wrapi((int)floor(rw[2] + 0.5), p->nz);
    if (is_solid(s, x, y, z)) return 0;
    node[0] = cell(s, x, y, z);
    w[0] = 1.0;
    return 1;
  }
  int x0[3];
  double sfrac[3];
  for (int a = 0; a < 3; ++a) {
    x0[a] = (int)floor(rw[a]);
    sfrac[a] = rw[a] - x0[a];
  }
  int n = 0;
  double wsum = 0;
  for (int k = 0; k < 8; ++k) {
    int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
    int x = wrapi(x0[0] + o[0], p->nx), y = wrapi(x0[1] + o[1], p->ny),
        z = wrapi(x0[2] + o[2], p->nz);
    if (is_solid(s, x, y, z)) continue;
    double wk = 1.0;
    for (int a = 0; a < 3; ++a) wk *= o[a] ? sfrac[a] : 1.0 - sfrac[a];
    node[n] = cell(s, x, y, z);
    w[n] = wk;
    wsum += wk;
    ++n;
  }
  if (n == 0 || wsum <= 0) return 0;
  for (int k = 0; k < n; ++k) w[k] /= wsum;
  return n;
}

/* u(x) -> u_i, from the moment field of the current f. */
static void gather(const orc_sim *s, const double *pos, double *ui) {
  const int64_t V = s->V;
  for (int i = 0; i < s->p.n_beads; ++i) {
    int64_t node[8];
    double w[8];
    int n = transfer_weights(s, &pos[3 * i], node, w);
    for (int a = 0; a < 3; ++a) {
      double acc = 0;
      for (int k = 0; k < n; ++k) acc += w[k] * s->u[a * V + node[k]];
      ui[3 * i + a] = acc;
    }
  }
}

/* F_i -> F(x): the fluid receives -J_i with the gather weights. */
static void spread(const orc_sim *s, const double *pos, const double *J,
                   double *F) {
  const int64_t V = s->V;
  memset(F, 0, sizeof(double) * 3 * V);
  for (int i = 0; i < s->p.n_beads; ++i) {
    int64_t node[8];
    double w[8];
    int n = transfer_weights(s, &pos[3 * i], node, w);
    for (int k = 0; k < n; ++k)
      for (int a = 0; a < 3; ++a) F[a * V + node[k]] -= w[k] * J[3 * i + a];
  }
}

/* ------------------------------------------------------------------ */
/* Bead forces (Eqs. 1-3 plus wall and drive)                          */
/* ------------------------------------------------------------------ */
static void min_image(const orc_params *p, double d[3]) {
  double L[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; ++a) d[a] -= L[a] * floor(d[a] / L[a] + 0.5);
}

static int bonded(const orc_sim *s, int i, int j) {
  for (int b = 0; b < s->p.n_bonds; ++b)
    if ((s->bi[b] == i && s->bj[b] == j) || (s->bi[b] == j && s->bj[b] == i))
      return 1;
  return 0;
}

/* Eq. 2 truncated at 2^(1/6) sigma and shifted by +eps (energy only).
 * Returns V; adds -dV/dd to Fout for separation vector d. */
static double wca(const orc_params *p, const double d[3], double Fout[3]) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double rc = pow(2.0, 1.0 / 6.0) * p->lj_sigma;
  if (r2 >= rc * rc) return 0.0;
  double sr2 = p->lj_sigma * p->lj_sigma / r2;
  double sr6 = sr2 * sr2 * sr2, sr12 = sr6 * sr6;
  double fmag_over_r = 24.0 * p->lj_eps * (2.0 * sr12 - sr6) / r2;
  for (int a = 0; a < 3; ++a) Fout[a] += fmag_over_r * d[a];
  return 4.0 * p->lj_eps * (sr12 - sr6) + p->lj_eps;
}

/* Eq. 3: V = kappa phi^2 / 2 with phi the angle between consecutive bonds
 * b1 = r_i - r_{i-1} and b2 = r_{i+1} - r_i of a linear chain.  Adds the
 * forces on beads i-1, i, i+1. */
static double bending(const orc_params *p, const double *pos, int i, double *F) {
  const double *ra = &pos[3 * (i - 1)], *rb = &pos[3 * i], *rc = &pos[3 * (i + 1)];
  double b1[3], b2[3];
  for (int a = 0; a < 3; ++a) {
    b1[a] = rb[a] - ra[a];
    b2[a] = rc[a] - rb[a];
  }
  double l1 = sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]);
  double l2 = sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
  double cphi = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) / (l1 * l2);
  if (cphi > 1.0) cphi = 1.0;
  if (cphi < -1.0) cphi = -1.0;
  double phi = acos(cphi);
  double sphi = sin(phi);
  /* dV/dcos(phi) = kappa phi dphi/dcos = -kappa phi / sin(phi) = -A */
  double A = (phi < 1e-8) ? p->kappa_phi : p->kappa_phi * phi / sphi;
  for (int a = 0; a < 3; ++a) {
    double g1 = b2[a] / (l1 * l2) - cphi * b1[a] / (l1 * l1); /* dcos/db1 */
    double g2 = b1[a] / (l1 * l2) - cphi * b2[a] / (l2 * l2); /* dcos/db2 */
    /* F = -dV/dr = A dcos/dr ; b1 = r_i - r_{i-1}, b2 = r_{i+1} - r_i */
    F[3 * (i - 1) + a] += -A * g1;
    F[3 * i + a] += A * (g1 - g2);
    F[3 * (i + 1) + a] += A * g2;
  }
  return 0.5 * p->kappa_phi * phi * phi;
}

/* Eq. 2 between a bead and every solid node closer than the cutoff. */
static double wall_force(const orc_sim *s, const double r[3], double Fo[3]) {
  const orc_params *p = &s->p;
  double rc = pow(2.0, 1.0 / 6.0) * p->lj_sigma;
  double L[3] = {p->nx, p->ny, p->nz};
  double rw[3];
  for (int a = 0; a < 3; ++a) rw[a] = wrapd(r[a], L[a]);
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = (int)ceil(rw[a] - rc);
    hi[a] = (int)floor(rw[a] + rc);
  }
  double E = 0;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        if (!is_solid(s, x, y, z)) continue;
        double d[3] = {rw[0] - x, rw[1] - y, rw[2] - z};
        E += wca(p, d, Fo);
      }
  return E;
}

/* Pulling force of Sec. III: -f_drive along x inside the channel formed by
 * the pore cross-section and the three x-layers centred on the wall
 * (|x - x_wall| <= 1.5 for a one-node wall). */
static void drive_force(const orc_sim *s, const double r[3], double Fo[3]) {
  const orc_params *p = &s->p;
  if (p->wall_x < 0 || p->pore_d <= 0 || p->f_drive == 0) return;
  int y0, z0;
  pore_origin(p, &y0, &z0);
  double xc = p->wall_x + 0.5 * (p->wall_thickness - 1);
  double half = 0.5 * (p->wall_thickness - 1) + 1.5;
  double dx = r[0] - xc;
  dx -= p->nx * floor(dx / p->nx + 0.5);
  double ry = wrapd(r[1], p->ny), rz = wrapd(r[2], p->nz);
  if (fabs(dx) <= half && ry >= y0 - 0.5 && ry < y0 + p->pore_d - 0.5 &&
      rz >= z0 - 0.5 && rz < z0 + p->pore_d - 0.5)
    Fo[0] -= p->f_drive;
}

/* Conservative + external forces on all beads at positions pos. */
static double conservative_forces(const orc_sim *s, const double *pos, double *F) {
  const orc_params *p = &s->p;
  int N = p->n_beads;
  double E = 0;
  memset(F, 0, sizeof(double) * 3 * N);
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      if (bonded(s, i, j)) continue;
      double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                     pos[3 * i + 2] - pos[3 * j + 2]};
      min_image(p, d);
      double f[3] = {0, 0, 0};
      E += wca(p, d, f);
      for (int a = 0; a < 3; ++a) {
        F[3 * i + a] += f[a];
        F[3 * j + a] -= f[a];
      }
    }
  if (p->kappa_phi != 0)
    for (int i = 1; i + 1 < N; ++i) E += bending(p, pos, i, F);
  for (int i = 0; i < N; ++i) {
    E += wall_force(s, &pos[3 * i], &F[3 * i]);
    drive_force(s, &pos[3 * i], &F[3 * i]);
  }
  return E;
}

/* ------------------------------------------------------------------ */
/* SHAKE (Ryckaert, Ciccotti, Berendsen 1977): Gauss-Seidel sweeps over  */
/* the bonds; each correction acts along the bond vector of the previous */
/* (constrained) positions.                                             */
/* ------------------------------------------------------------------ */
static int shake(const orc_sim *s, const double *r_old, double *r_new,
                 int *sweeps_out) {
  const orc_params *p = &s->p;
  double im = 1.0 / p->mass;
  int sweep;
  for (sweep = 0; sweep < p->shake_max_iter; ++sweep) {
    double maxerr = 0;
    for (int b = 0; b < p->n_bonds; ++b) {
      int i = s->bi[b], j = s->bj[b];
      double sb[3], d[3];
      for (int a = 0; a < 3; ++a) {
        sb[a] = r_old[3 * j + a] - r_old[3 * i + a];
        d[a] = r_new[3 * j + a] - r_new[3 * i + a];
      }
      double diff = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - s->b0[b] * s->b0[b];
      double err = fabs(diff) / (s->b0[b] * s->b0[b]);
      if (err > maxerr) maxerr = err;
      double sd = sb[0] * d[0] + sb[1] * d[1] + sb[2] * d[2];
      double gfac = diff / (2.0 * sd * (im + im));
      for (int a = 0; a < 3; ++a) {
        r_new[3 * i + a] += gfac * sb[a] * im;
        r_new[3 * j + a] -= gfac * sb[a] * im;
      }
    }
    if (!(maxerr == maxerr)) break; /* NaN */
    if (maxerr < p->shake_tol) {
      *sweeps_out = sweep + 1;
      return 0;
    }
  }
  *sweeps_out = sweep;
  return -1;
}

/* RATTLE velocity stage (Andersen 1983): remove the relative velocity along
 * every bond, Gauss-Seidel. */
static int rattle(const orc_sim *s, const double *r, double *v, int *sweeps_out) {
  const orc_params *p = &s->p;
  double im = 1.0 / p->mass;
  int sweep;
  for (sweep = 0; sweep < p->shake_max_iter; ++sweep) {
    double maxerr = 0;
    for (int b = 0; b < p->n_bonds; ++b) {
      int i = s->bi[b], j = s->bj[b];
      double d[3], dv[3];
      for (int a = 0; a < 3; ++a) {
        d[a] = r[3 * j + a] - r[3 * i + a];
        dv[a] = v[3 * j + a] - v[3 * i + a];
      }
      double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      double proj = d[0] * dv[0] + d[1] * dv[1] + d[2] * dv[2];
      if (fabs(proj) > maxerr) maxerr = fabs(proj);
      double k = proj / (dd * (im + im));
      for (int a = 0; a < 3; ++a) {
        v[3 * i + a] += k * d[a] * im;
        v[3 * j + a] -= k * d[a] * im;
      }
    }
    if (!(maxerr == maxerr)) break;
    if (maxerr < p->shake_tol) {
      *sweeps_out = sweep + 1;
      return 0;
    }
  }
  *sweeps_out = sweep;
  return -1;
}

/* ------------------------------------------------------------------ */
/* One MD substep of length dt_MD = 1/M with u_i frozen (Sec. II).      */
/* ------------------------------------------------------------------ */
static int md_substep(orc_sim *s, int k, double *Fc, double *rnew) {
  const orc_params *p = &s->p;
  int N = p->n_beads;
  double dt = 1.0 / p->md_substeps;
  double m = p->mass;
  double sig_r = sqrt(2.0 * m * p->gamma * p->kT / dt);
  conservative_forces(s, s->r, Fc);
  for (int i = 0; i < N; ++i) {
    double xi[3];
    orc_gauss3(p->seed, (uint32_t)i, s->step, (uint32_t)k, 0u, xi);
    for (int a = 0; a < 3; ++a) {
      double fdrag = -m * p->gamma * (s->v[3 * i + a] - s->ui[3 * i + a]);
      double frand = sig_r * xi[a];
      double vnew = s->v[3 * i + a] + dt * (Fc[3 * i + a] + fdrag + frand) / m;
      /* impulse handed to the fluid (after the substep loop) */
      s->J[3 * i + a] += dt * (fdrag + frand);
      s->v[3 * i + a] = vnew;
      rnew[3 * i + a] = s->r[3 * i + a] + dt * vnew;
    }
  }
  int sweeps = 0, rc = 0;
  if (p->n_bonds > 0) {
    if (shake(s, s->r, rnew, &sweeps) != 0) rc = -1;
    s->last_shake_sweeps = sweeps;
  }
  for (int i = 0; i < 3 * N; ++i) {
    s->v[i] = (rnew[i] - s->r[i]) / dt;
    s->r[i] = rnew[i];
  }
  if (p->n_bonds > 0) {
    if (rattle(s, s->r, s->v, &sweeps) != 0) rc = -1;
    s->last_rattle_sweeps = sweeps;
  }
  return rc;
}

/* Translocation bookkeeping (Sec. III): N_T counts beads on the trans side
 * x < x_wall (unwrapped x); completion at N_T = N; retraction when, after at
 * least one bead crossed, every bead is back beyond the drive channel. */
static void bookkeeping(orc_sim *s, int shake_rc) {
  const orc_params *p = &s->p;
  int N = p->n_beads;
  int nan = 0;
  for (int i = 0; i < 3 * N; ++i)
    if (!isfinite(s->r[i]) || !isfinite(s->v[i])) nan = 1;
  int nt = 0;
  double xmin = INFINITY;
  if (p->wall_x >= 0)
    for (int i = 0; i < N; ++i) {
      if (s->r[3 * i] < p->wall_x) ++nt;
      if (s->r[3 * i] < xmin) xmin = s->r[3 * i];
    }
  s->n_trans = nt;
  if (nt > s->max_trans) s->max_trans = nt;
  if (s->state != ORC_RUNNING) return;
  if (nan) {
    s->state = ORC_NAN;
    return;
  }
  if (shake_rc != 0) {
    s->state = ORC_SHAKE_FAIL;
    return;
  }
  if (p->wall_x < 0 || N == 0) return;
  if (nt == N) {
    s->state = ORC_TRANSLOCATED;
    s->t_transloc = s->step;
  } else if (s->max_trans >= 1 &&
             xmin > p->wall_x + (p->wall_thickness - 1) + 1.5) {
    s->state = ORC_RETRACTED;
  }
}

/* One LB step: the four stages of the Sec. II scheme. */
static int one_step(orc_sim *s, double *Fc, double *rnew, double *r_start) {
  const orc_params *p = &s->p;
  int N = p->n_beads;
  const int hydro = p->hydrodynamics;
  if (hydro) compute_moments(s);
  int shake_rc = 0;
  if (N > 0) {
    /* (i) interpolation of the fluid velocity to the beads */
    if (hydro)
      gather(s, s->r, s->ui);
    else
      memset(s->ui, 0, sizeof(double) * 3 * N);
    memcpy(r_start, s->r, sizeof(double) * 3 * N);
    memset(s->J, 0, sizeof(double) * 3 * N);
    /* (ii) M MD substeps with the hydrodynamic field frozen */
    for (int k = 0; k < p->md_substeps; ++k)
      if (md_substep(s, k, Fc, rnew) != 0) shake_rc = -1;
    /* (iii) extrapolation of the forces to the grid */
    if (hydro) spread(s, r_start, s->J, s->F);
  } else {
    memset(s->F, 0, sizeof(double) * 3 * s->V);
  }
  /* (iv) advance the populations */
  if (hydro) {
    collide_all(s);
    stream_all(s);
  }
  s->step += 1;
  bookkeeping(s, shake_rc);
  return shake_rc;
}

int orc_step(orc_sim *s, int64_t n) {
  int N = s->p.n_beads;
  size_t nn = (size_t)(3 * (N > 0 ? N : 1));
  double *Fc = (double *)calloc(nn, sizeof(double));
  double *rnew = (double *)calloc(nn, sizeof(double));
  double *r_start = (double *)calloc(nn, sizeof(double));
  int rc = 0;
  if (!Fc || !rnew || !r_start) rc = -2;
  for (int64_t t = 0; t < n && rc != -2; ++t)
    if (one_step(s, Fc, rnew, r_start) != 0) rc = -1;
  free(Fc);
  free(rnew);
  free(r_start);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Read-outs and single-stage entry points for the pin tests           */
/* ------------------------------------------------------------------ */
void orc_get_populations(const orc_sim *s, double *f) {
  memcpy(f, s->f, sizeof(double) * Q * s->V);
}
void orc_set_populations(orc_sim *s, const double *f) {
  memcpy(s->f, f, sizeof(double) * Q * s->V);
}
void orc_get_fields(orc_sim *s, double *rho, double *u) {
  compute_moments(s);
  memcpy(rho, s->rho, sizeof(double) * s->V);
  memcpy(u, s->u, sizeof(double) * 3 * s->V);
}
void orc_get_beads(const orc_sim *s, double *pos, double *vel) {
  memcpy(pos, s->r, sizeof(double) * 3 * s->p.n_beads);
  memcpy(vel, s->v, sizeof(double) * 3 * s->p.n_beads);
}
void orc_set_beads(orc_sim *s, const double *pos, const double *vel) {
  memcpy(s->r, pos, sizeof(double) * 3 * s->p.n_beads);
  memcpy(s->v, vel, sizeof(double) * 3 * s->p.n_beads);
}
void orc_get_bead_aux(const orc_sim *s, double *ui, double *J) {
  memcpy(ui, s->ui, sizeof(double) * 3 * s->p.n_beads);
  memcpy(J, s->J, sizeof(double) * 3 * s->p.n_beads);
}
void orc_get_force_field(const orc_sim *s, double *F) {
  memcpy(F, s->F, sizeof(double) * 3 * s->V);
}
void orc_get_solid(const orc_sim *s, uint8_t *solid) {
  memcpy(solid, s->solid, (size_t)s->V);
}
void orc_get_status(const orc_sim *s, int64_t *step, int32_t *n_trans,
                    int32_t *state, int64_t *t_transloc) {
  *step = s->step;
  *n_trans = s->n_trans;
  *state = s->state;
  *t_transloc = s->t_transloc;
}
void orc_get_sweeps(const orc_sim *s, int32_t *shake_sweeps,
                    int32_t *rattle_sweeps) {
  *shake_sweeps = s->last_shake_sweeps;
  *rattle_sweeps = s->last_rattle_sweeps;
}
double orc_forces(orc_sim *s, const double *pos, double *F) {
  return conservative_forces(s, pos, F);
}
void orc_gather(orc_sim *s, const double *pos, double *ui) {
  compute_moments(s);
  gather(s, pos, ui);
}
void orc_spread(const orc_sim *s, const double *pos, const double *J, double *F) {
  spread(s, pos, J, F);
}
int orc_transfer_weights(const orc_sim *s, const double r[3], int64_t node[8],
                         double w[8]) {
  return transfer_weights(s, r, node, w);
}
int orc_shake(const orc_sim *s, const double *r_old, double *r_new, int32_t *sweeps) {
  int sw = 0;
  int rc = shake(s, r_old, r_new, &sw);
  *sweeps = sw;
  return rc;
}
int orc_rattle(const orc_sim *s, const double *r, double *v, int32_t *sweeps) {
  int sw = 0;
  int rc = rattle(s, r, v, &sw);
  *sweeps = sw;
  return rc;
}
/* Chain diagnostics of Sec. III at bead positions r (unwrapped), velocities
 * v and interpolated fluid velocities ui (3*N each):
 *   out[0] R_U, out[1] R_T: radii of gyration of the untranslocated
 *          (x >= x_wall) and translocated (x < x_wall) beads, 0 for an
 *          empty part;
 *   out[2] R_E = (R_T^(1/mu) + R_U^(1/mu))^mu, mu = 0.6;
 *   out[3] S_H = m gamma sum_i v_i . u_i (Eq. 13, the fluid's work rate;
 *          the paper's unit mass);
 *   out[4] S_E = sum_i F_drive(r_i) . v_i (Eq. 14);
 *   out[5] K = m/2 sum_i |v_i|^2;
 *   out[6] N_T.
 * Without a wall every bead counts as untranslocated. */
void orc_diagnostics(const orc_sim *s, const double *r, const double *v, const double *ui,
                     double out[7]) {
  const orc_params *p = &s->p;
  const int N = p->n_beads;
  double cm[2][3] = {{0, 0, 0}, {0, 0, 0}};
  int cnt[2] = {0, 0};
  for (int i = 0; i < N; ++i) {
    const int t = (p->wall_x >= 0 && r[3 * i] < p->wall_x) ? 1 : 0;
    cnt[t] += 1;
    for (int a = 0; a < 3; ++a) cm[t][a] += r[3 * i + a];
  }
  for (int t = 0; t < 2; ++t)
    for (int a = 0; a < 3; ++a) cm[t][a] = cnt[t] ? cm[t][a] / cnt[t] : 0.0;
  double r2[2] = {0, 0};
  double sh = 0, se = 0, ke = 0;
  for (int i = 0; i < N; ++i) {
    const int t = (p->wall_x >= 0 && r[3 * i] < p->wall_x) ? 1 : 0;
    double Fd[3] = {0, 0, 0};
    drive_force(s, &r[3 * i], Fd);
    for (int a = 0; a < 3; ++a) {
      const double d = r[3 * i + a] - cm[t][a];
      r2[t] += d * d;
      sh += v[3 * i + a] * ui[3 * i + a];
      se += Fd[a] * v[3 * i + a];
      ke += v[3 * i + a] * v[3 * i + a];
    }
  }
  const double mu = 0.6;
  const double RU = cnt[0] ? sqrt(r2[0] / cnt[0]) : 0.0;
  const double RT = cnt[1] ? sqrt(r2[1] / cnt[1]) : 0.0;
  out[0] = RU;
  out[1] = RT;
  out[2] = pow(pow(RT, 1.0 / mu) + pow(RU, 1.0 / mu), mu);
  out[3] = p->mass * p->gamma * sh;
  out[4] = se;
  out[5] = 0.5 * p->mass * ke;
  out[6] = cnt[1];
}

void orc_state_diagnostics(const orc_sim *s, double out[7]) {
  orc_diagnostics(s, s->r, s->v, s->ui, out);
}

int orc_weights_table(double w[Q], int32_t c[3 * Q]) {
  for (int p = 0; p < Q; ++p) {
    w[p] = weight(p);
    for (int a = 0; a < 3; ++a) c[3 * p + a] = CV[p][a];
  }
  return Q;
}
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
