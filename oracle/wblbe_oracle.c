/*
 * FP64 CPU oracle for the standard LBE (Sec. II) and the well-balanced LBE
 * (Sec. III) of Guo, "Well-balanced lattice Boltzmann equation for two-phase
 * flows" (arXiv 2012.11075).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Conventions (all from the paper unless marked "reading"):
 *   - lattice units dx = dt = c = 1, cs^2 = 1/3 (Sec. II, after Eq. D2Q9);
 *   - D2Q9 velocities c0=(0,0), c1=-c3=(1,0), c2=-c4=(0,1), c5=-c7=(1,1),
 *     c6=-c8=(-1,1) (Sec. II; the printed "c7=-c8" is read as c6=-c8, the
 *     only numbering that leaves nine distinct velocities);
 *   - weights 4/9, 1/9 (x4), 1/36 (x4) (Sec. II, after Eq. feq);
 *   - BGK update f_i(x+c_i,t+1) = f_i - (f_i - f_i^eq)/tau + (1 - 1/(2 tau)) F_i
 *     (Eq. D2Q9; the printed "+1/tau" is read as the usual relaxation sign,
 *     the one under which the paper's own steady-state relation
 *     f_i = f_i^eq + (tau - 1/2) F_i for group A holds);
 *   - periodic boundaries in x and y (Sec. IV);
 *   - populations stored as f[i][y][x] (x fastest), nine planes of nx*ny.
 *
 * Discretisations the paper does not print (reading): the gradient is the
 * isotropic central scheme  grad(phi) = (1/cs^2) sum_i w_i c_i phi(x+c_i),
 * which reduces to (phi_{j+1}-phi_{j-1})/2 in 1D as Sec. II states; the
 * Laplacian is the matching isotropic form
 * lap(phi) = (2/cs^2) sum_i w_i (phi(x+c_i) - phi(x)).
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused: the
 * arithmetic is exactly the order written here on every host.
 *
 * The "omp parallel for" lines split loops whose iterations write disjoint
 * memory across threads; they are ignored unless the file is built with
 * -fopenmp, which only the timing build of the benchmark's all-cores CPU
 * baseline does.  Every node is computed the same way either way.
 *
 * Built with -DORC_DENSITY_PAIRWISE (a rounding-sensitivity build, used only
 * by tests), the density rho = sum_i f_i is summed in pairs instead of from
 * i = 0 to 8.  Nothing else changes: comparing the two builds measures how
 * far two equally valid FP64 evaluations of the same update drift apart.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define Q 9
#define DIM 2

static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* Schemes: the standard LBE of Sec. II (potential-form force, Eq. Fi), the
 * well-balanced LBE of Sec. III, and variants of the standard LBE that
 * Sec. II compares it with: the pressure-form force; the forcing term of
 * Guo's textbook, F_i = (c_i - u).F f_i^eq / (cs^2 rho); and a higher-order
 * gradient for the force (ORC_STANDARD_E6, see orc_gradient6). */
enum { ORC_STANDARD = 0, ORC_WELL_BALANCED = 1, ORC_STANDARD_PRESSURE = 2,
       ORC_STANDARD_TEXTBOOK = 3, ORC_STANDARD_E6 = 4 };

/* Problem statement (Sec. IV): lattice, relaxation time, free-energy
 * parameters, the WB constant rho0 (Eq. mFeq) and the scheme. */
typedef struct {
  int nx, ny;
  double tau, kappa, beta, rho_l, rho_g, rho0;
  int scheme;
} orc_params;

typedef struct {
  double mass, umax, mu_min, mu_max, kinetic;
  int nonfinite;
} orc_stats;

/* Periodic index for a in [-n, 2n): every use below is a node index plus a
 * lattice offset of -1, 0 or +1. */
static int wrap(int a, int n) {
  if (a < 0) return a + n;
  if (a >= n) return a - n;
  return a;
}

static size_t node(const orc_params* p, int x, int y) {
  return (size_t)wrap(y, p->ny) * (size_t)p->nx + (size_t)wrap(x, p->nx);
}

/* ---- Free energy, Eq. doubleWell and Eq. EOS ---------------------------- */

/* psi_0 = beta (rho - rho_l)^2 (rho - rho_v)^2 */
double orc_psi0(const orc_params* p, double rho) {
  double a = rho - p->rho_l, b = rho - p->rho_g;
  return p->beta * a * a * b * b;
}

/* mu_0 = d psi_0 / d rho, written as the product rule applied to psi_0. */
double orc_mu0(const orc_params* p, double rho) {
  double a = rho - p->rho_l, b = rho - p->rho_g;
  return 2.0 * p->beta * a * b * b + 2.0 * p->beta * a * a * b;
}

/* p_0 = rho dpsi_0/drho - psi_0 (Eq. EOS; the printed form lacks the factor
 * rho, which the thermodynamic identity p = rho mu - psi requires). */
double orc_p0(const orc_params* p, double rho) {
  return rho * orc_mu0(p, rho) - orc_psi0(p, rho);
}

/* ---- Finite-difference operators (isotropic central scheme) ------------- */

/* lap(phi)(x) = (2/cs^2) sum_i w_i (phi(x+c_i) - phi(x)) */
void orc_laplacian(const orc_params* p, const double* phi, double* out) {
#pragma omp parallel for
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      double s = 0.0;
      double c = phi[node(p, x, y)];
      for (int i = 0; i < Q; ++i)
        s += WQ[i] * (phi[node(p, x + CX[i], y + CY[i])] - c);
      out[node(p, x, y)] = 2.0 / CS2 * s;
    }
}

/* grad(phi)(x) = (1/cs^2) sum_i w_i c_i phi(x+c_i) */
void orc_gradient(const orc_params* p, const double* phi, double* gx,
                  double* gy) {
#pragma omp parallel for
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      double sx = 0.0, sy = 0.0;
      for (int i = 0; i < Q; ++i) {
        double v = phi[node(p, x + CX[i], y + CY[i])];
        sx += WQ[i] * CX[i] * v;
        sy += WQ[i] * CY[i] * v;
      }
      gx[node(p, x, y)] = sx / CS2;
      gy[node(p, x, y)] = sy / CS2;
    }
}

/* Higher-order isotropic gradient for the force of ORC_STANDARD_E6.  Sec. II
 * notes that higher-order discretisations of F reduce the spurious velocity
 * but cannot balance the forces; it names no stencil (reading: the
 * radius-2 gradient whose weights make the lattice moments isotropic up to
 * sixth order).  grad(phi) = sum_e W(|e|^2) e phi(x+e) over the shells
 * |e|^2 = 1 (4 vectors), 2 (4) and 4 (4: (+-2,0), (0,+-2)); the weights solve
 *   sum W e_x^2 = 1                 (exact on linear functions),
 *   sum W e_x^4 = 3 sum W e_x^2 e_y^2  (4th-order moments isotropic),
 *   sum W e_x^6 = 5 sum W e_x^4 e_y^2  (6th-order moments isotropic),
 * i.e. 2W1 + 4W2 + 8W4 = 1, 2W1 - 8W2 + 32W4 = 0, 2W1 - 16W2 + 128W4 = 0:
 * W1 = 4/15, W2 = 1/10, W4 = 1/120.  (The 9-point gradient above is the
 * 4th-order case: W1 = 1/3, W2 = 1/12.) */
static const double W6_1 = 4.0 / 15.0, W6_2 = 1.0 / 10.0, W6_4 = 1.0 / 120.0;

void orc_gradient6(const orc_params* p, const double* phi, double* gx, double* gy) {
  static const int EX[12] = {1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0};
  static const int EY[12] = {0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2};
#pragma omp parallel for
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      double sx = 0.0, sy = 0.0;
      for (int a = 0; a < 12; ++a) {
        double w = a < 4 ? W6_1 : (a < 8 ? W6_2 : W6_4);
        /* offsets up to 2: wrap twice */
        int xx = x + EX[a], yy = y + EY[a];
        xx = (xx % p->nx + p->nx) % p->nx;
        yy = (yy % p->ny + p->ny) % p->ny;
        double v = phi[(size_t)yy * (size_t)p->nx + (size_t)xx];
        sx += w * EX[a] * v;
        sy += w * EY[a] * v;
      }
      gx[node(p, x, y)] = sx;
      gy[node(p, x, y)] = sy;
    }
}

/* ---- Equilibria and forcing terms, per node ----------------------------- */

/* Standard equilibrium, Eq. feq (the printed signs of the two quadratic
 * terms are read as the usual second-order expansion, the one that gives the
 * paper's group-A relation f_A = (2/3) rho (1 - v^2/(2cs^2)) + ...). */
static void feq_standard(double rho, double ux, double uy, double* feq) {
  double uu = ux * ux + uy * uy;
  for (int i = 0; i < Q; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    feq[i] = WQ[i] * rho *
             (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
  }
}

/* Well-balanced equilibrium, Eq. mFeq. */
static void feq_well_balanced(double rho, double ux, double uy, double rho0,
                              double* feq) {
  double uu = ux * ux + uy * uy;
  feq[0] = rho - (1.0 - WQ[0]) * rho0 - WQ[0] * rho * uu / (2.0 * CS2);
  for (int i = 1; i < Q; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    feq[i] = WQ[i] * (rho0 + rho * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) -
                                    uu / (2.0 * CS2)));
  }
}

/* u a : (c_i c_i - cs^2 I), the double contraction written out. */
static double contract(int i, double ux, double uy, double ax, double ay) {
  double u[DIM] = {ux, uy}, a[DIM] = {ax, ay};
  double c[DIM] = {(double)CX[i], (double)CY[i]};
  double s = 0.0;
  for (int al = 0; al < DIM; ++al)
    for (int be = 0; be < DIM; ++be)
      s += u[al] * a[be] * (c[al] * c[be] - (al == be ? CS2 : 0.0));
  return s;
}

/* Standard forcing term, Eq. Fi. */
static void forcing_standard(double ux, double uy, double Fx, double Fy,
                             double* Fi) {
  for (int i = 0; i < Q; ++i) {
    double cF = CX[i] * Fx + CY[i] * Fy;
    Fi[i] = WQ[i] * (cF / CS2 + contract(i, ux, uy, Fx, Fy) / (CS2 * CS2));
  }
}

/* Well-balanced forcing term, Eq. mFi, D = 2. */
static void forcing_well_balanced(double ux, double uy, double Fx, double Fy,
                                  double grx, double gry, double* Fi) {
  double Gx = Fx + CS2 * grx, Gy = Fy + CS2 * gry;
  double ugr = ux * grx + uy * gry;
  for (int i = 0; i < Q; ++i) {
    double cF = CX[i] * Fx + CY[i] * Fy;
    double c2 = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
    Fi[i] = WQ[i] * (cF / CS2 + contract(i, ux, uy, Gx, Gy) / (CS2 * CS2) +
                     0.5 * (c2 / CS2 - DIM) * ugr);
  }
}

/* Forcing term of Guo's textbook quoted in Sec. II:
 * F_i = (c_i - u).F f_i^eq / (cs^2 rho), with the standard equilibrium; the
 * density cancels, f_i^eq / rho being the standard equilibrium at rho = 1. */
static void forcing_guo_book(double ux, double uy, double Fx, double Fy,
                             double* Fi) {
  double feq1[Q];
  feq_standard(1.0, ux, uy, feq1);
  for (int i = 0; i < Q; ++i) {
    double cuF = (CX[i] - ux) * Fx + (CY[i] - uy) * Fy;
    Fi[i] = cuF * feq1[i] / CS2;
  }
}

void orc_feq(const orc_params* p, double rho, double ux, double uy,
             double* feq) {
  if (p->scheme == ORC_WELL_BALANCED)
    feq_well_balanced(rho, ux, uy, p->rho0, feq);
  else
    feq_standard(rho, ux, uy, feq);
}

void orc_forcing(const orc_params* p, double ux, double uy, double Fx,
                 double Fy, double grx, double gry, double* Fi) {
  if (p->scheme == ORC_WELL_BALANCED)
    forcing_well_balanced(ux, uy, Fx, Fy, grx, gry, Fi);
  else if (p->scheme == ORC_STANDARD_TEXTBOOK)
    forcing_guo_book(ux, uy, Fx, Fy, Fi);
  else
    forcing_standard(ux, uy, Fx, Fy, Fi);
}

/* ---- Macroscopic fields of a population state --------------------------- */

/* Given f (post-streaming, pre-collision), compute
 *   rho = sum_i f_i                                  (Eq. rhoU)
 *   mu  = mu_0(rho) - kappa lap(rho)                 (Sec. II)
 *   F   = -rho grad(mu)                 (WB, Eq. mF)
 *       = grad(cs^2 rho) - rho grad(mu) (standard, potential form, Sec. II)
 *       = grad(cs^2 rho - p_0) + kappa rho grad(lap(rho))
 *                                       (standard, pressure form, Sec. II)
 * The pressure form is printed with "- kappa grad(lap rho)"; the paper calls
 * the two forms identical, which holds only with "+ kappa rho grad(lap rho)"
 * (rho grad mu = grad p_0 - kappa rho grad lap rho, from p_0 = rho mu_0 -
 * psi_0): that is the reading taken.
 *   u   = (sum_i c_i f_i + F/2) / rho                (Eq. rhoU)
 * Any output pointer may be NULL. */
void orc_macro(const orc_params* p, const double* f, double* rho_out,
               double* mu_out, double* ux_out, double* uy_out, double* Fx_out,
               double* Fy_out, double* grx_out, double* gry_out) {
  size_t n = (size_t)p->nx * (size_t)p->ny;
  double* rho = (double*)malloc(n * sizeof(double));
  double* lap = (double*)malloc(n * sizeof(double));
  double* mu = (double*)malloc(n * sizeof(double));
  double* gmx = (double*)malloc(n * sizeof(double));
  double* gmy = (double*)malloc(n * sizeof(double));
  double* grx = (double*)malloc(n * sizeof(double));
  double* gry = (double*)malloc(n * sizeof(double));

#pragma omp parallel for
  for (size_t k = 0; k < n; ++k) {
#ifdef ORC_DENSITY_PAIRWISE
    const double* g = f + k;
    rho[k] = ((g[0] + g[n]) + (g[2 * n] + g[3 * n])) +
             ((g[4 * n] + g[5 * n]) + (g[6 * n] + g[7 * n])) + g[8 * n];
#else
    double s = 0.0;
    for (int i = 0; i < Q; ++i) s += f[(size_t)i * n + k];
    rho[k] = s;
#endif
  }
  orc_laplacian(p, rho, lap);
#pragma omp parallel for
  for (size_t k = 0; k < n; ++k) mu[k] = orc_mu0(p, rho[k]) - p->kappa * lap[k];
  if (p->scheme == ORC_STANDARD_E6) {
    orc_gradient6(p, mu, gmx, gmy);
    orc_gradient6(p, rho, grx, gry);
  } else {
    orc_gradient(p, mu, gmx, gmy);
    orc_gradient(p, rho, grx, gry);
  }
  /* pressure form: gmx/gmy become grad(lap rho), and gAx/gAy the gradient of
   * A = cs^2 rho - p_0(rho) */
  double* gAx = NULL;
  double* gAy = NULL;
  if (p->scheme == ORC_STANDARD_PRESSURE) {
    double* A = (double*)malloc(n * sizeof(double));
    gAx = (double*)malloc(n * sizeof(double));
    gAy = (double*)malloc(n * sizeof(double));
    for (size_t k = 0; k < n; ++k) A[k] = CS2 * rho[k] - orc_p0(p, rho[k]);
    orc_gradient(p, A, gAx, gAy);
    orc_gradient(p, lap, gmx, gmy);
    free(A);
  }

#pragma omp parallel for
  for (size_t k = 0; k < n; ++k) {
    double Fx, Fy;
    if (p->scheme == ORC_WELL_BALANCED) {
      Fx = -rho[k] * gmx[k];
      Fy = -rho[k] * gmy[k];
    } else if (p->scheme == ORC_STANDARD_PRESSURE) {
      Fx = gAx[k] + p->kappa * rho[k] * gmx[k];
      Fy = gAy[k] + p->kappa * rho[k] * gmy[k];
    } else {
      Fx = CS2 * grx[k] - rho[k] * gmx[k];
      Fy = CS2 * gry[k] - rho[k] * gmy[k];
    }
    double jx = 0.0, jy = 0.0;
    for (int i = 0; i < Q; ++i) {
      jx += CX[i] * f[(size_t)i * n + k];
      jy += CY[i] * f[(size_t)i * n + k];
    }
    if (rho_out) rho_out[k] = rho[k];
    if (mu_out) mu_out[k] = mu[k];
    if (ux_out) ux_out[k] = (jx + 0.5 * Fx) / rho[k];
    if (uy_out) uy_out[k] = (jy + 0.5 * Fy) / rho[k];
    if (Fx_out) Fx_out[k] = Fx;
    if (Fy_out) Fy_out[k] = Fy;
    if (grx_out) grx_out[k] = grx[k];
    if (gry_out) gry_out[k] = gry[k];
  }
  free(rho); free(lap); free(mu); free(gmx); free(gmy); free(grx); free(gry);
  free(gAx); free(gAy);
}

/* ---- Initial state ------------------------------------------------------ */

/* f = f^eq(rho, u = 0), no forcing correction (Sec. IV: the runs start from
 * the density profile at rest). */
void orc_init(const orc_params* p, const double* rho, double* f) {
  size_t n = (size_t)p->nx * (size_t)p->ny;
  double feq[Q];
  for (size_t k = 0; k < n; ++k) {
    orc_feq(p, rho[k], 0.0, 0.0, feq);
    for (int i = 0; i < Q; ++i) f[(size_t)i * n + k] = feq[i];
  }
}

/* ---- One time step ------------------------------------------------------ */

/* f holds f_i(x, t); on return it holds f_i(x, t+1).  work must hold
 * 9*nx*ny + 8*nx*ny doubles. */
static void step_once(const orc_params* p, double* f, double* work) {
  size_t n = (size_t)p->nx * (size_t)p->ny;
  double* fnew = work;
  double* rho = work + (size_t)Q * n;
  double* mu = rho + n;
  double* ux = mu + n;
  double* uy = ux + n;
  double* Fx = uy + n;
  double* Fy = Fx + n;
  double* grx = Fy + n;
  double* gry = grx + n;
  double omega = 1.0 / p->tau;
  double kforce = 1.0 - 1.0 / (2.0 * p->tau);

  orc_macro(p, f, rho, mu, ux, uy, Fx, Fy, grx, gry);

#pragma omp parallel for
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      size_t k = node(p, x, y);
      double feq[Q], Fi[Q];
      orc_feq(p, rho[k], ux[k], uy[k], feq);
      orc_forcing(p, ux[k], uy[k], Fx[k], Fy[k], grx[k], gry[k], Fi);
      for (int i = 0; i < Q; ++i) {
        double fi = f[(size_t)i * n + k];
        double post = fi - omega * (fi - feq[i]) + kforce * Fi[i];
        /* streaming: the post-collision value moves to x + c_i */
        fnew[(size_t)i * n + node(p, x + CX[i], y + CY[i])] = post;
      }
    }
  memcpy(f, fnew, (size_t)Q * n * sizeof(double));
}

/* Advance nsteps time steps in place.  Returns 0, or -1 if out of memory. */
int orc_step(const orc_params* p, double* f, long nsteps) {
  size_t n = (size_t)p->nx * (size_t)p->ny;
  double* work = (double*)malloc((size_t)(Q + 8) * n * sizeof(double));
  if (!work) return -1;
  for (long s = 0; s < nsteps; ++s) step_once(p, f, work);
  free(work);
  return 0;
}

/* ---- Diagnostics (Sec. IV) ---------------------------------------------- */

/* mass = sum rho (compensated sum), max |u|, min/max mu,
 * kinetic energy E = 1/2 sum rho |u|^2, and a flag for any non-finite value. */
void orc_stats_of(const orc_params* p, const double* f, orc_stats* st) {
  size_t n = (size_t)p->nx * (size_t)p->ny;
  double* rho = (double*)malloc(n * sizeof(double));
  double* mu = (double*)malloc(n * sizeof(double));
  double* ux = (double*)malloc(n * sizeof(double));
  double* uy = (double*)malloc(n * sizeof(double));
  orc_macro(p, f, rho, mu, ux, uy, NULL, NULL, NULL, NULL);
  double sum = 0.0, comp = 0.0, umax = 0.0, e = 0.0;
  double mumin = INFINITY, mumax = -INFINITY;
  int bad = 0;
  for (size_t k = 0; k < n; ++k) {
    double yk = rho[k] - comp;
    double t = sum + yk;
    comp = (t - sum) - yk;
    sum = t;
    double um = sqrt(ux[k] * ux[k] + uy[k] * uy[k]);
    if (um > umax) umax = um;
    if (mu[k] < mumin) mumin = mu[k];
    if (mu[k] > mumax) mumax = mu[k];
    e += 0.5 * rho[k] * (ux[k] * ux[k] + uy[k] * uy[k]);
    if (!isfinite(rho[k]) || !isfinite(mu[k]) || !isfinite(ux[k]) ||
        !isfinite(uy[k]))
      bad = 1;
  }
  st->mass = sum;
  st->umax = umax;
  st->mu_min = mumin;
  st->mu_max = mumax;
  st->kinetic = e;
  st->nonfinite = bad;
  free(rho); free(mu); free(ux); free(uy);
}
