/*
 * FP64 CPU oracle for the three-dimensional form of the well-balanced LBE
 * (Sec. III of Guo, "Well-balanced lattice Boltzmann equation for two-phase
 * flows", arXiv 2012.11075) and of the standard LBE (Sec. II), on the D3Q19
 * lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * What the paper fixes, in any dimension D: the update of Eq. D2Q9 (BGK
 * relaxation plus the forcing term, streaming along c_i), rho and u of
 * Eq. rhoU, the well-balanced equilibrium of Eq. mFeq, the force
 * F = -rho grad(mu) of Eq. mF and the forcing term of Eq. mFi, whose last
 * term carries the dimension D explicitly; Sec. V says the construction
 * carries over to other lattice Boltzmann models.  The standard scheme of
 * Sec. II (Eq. feq, the potential-form force, Eq. Fi) likewise.
 *
 * Readings (the paper works on D2Q9 only):
 *   - lattice: D3Q19, c_0 = 0; the six axis vectors (+-1,0,0), (0,+-1,0),
 *     (0,0,+-1) with w = 1/18; the twelve edge vectors (+-1,+-1,0),
 *     (+-1,0,+-1), (0,+-1,+-1) with w = 1/36; w_0 = 1/3; cs^2 = 1/3;
 *   - D = 3 in Eq. mFi;
 *   - the isotropic central stencils of the 2D oracle with these weights:
 *     grad(phi) = (1/cs^2) sum_i w_i c_i phi(x+c_i),
 *     lap(phi)  = (2/cs^2) sum_i w_i (phi(x+c_i) - phi(x)),
 *     which reduce to the 1D central forms on a field that varies along one
 *     axis only;
 *   - collision sign, initial state and free energy as in the 2D oracle.
 *
 * Populations are stored as f[i][z][y][x] (x fastest).  Compile with
 * -ffp-contract=off: the arithmetic is exactly the order written here.
 * Built with -DORC_DENSITY_PAIRWISE (tests only), rho = sum_i f_i is summed
 * in pairs instead of in sequence, nothing else changed: the spread between
 * the two builds measures the FP64 conditioning of the update.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define Q3 19
#define D3 3

static const int EX[Q3] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[Q3] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[Q3] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
static double WQ3(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
static const double CS2_3 = 1.0 / 3.0;

enum { O3_STANDARD = 0, O3_WELL_BALANCED = 1 };

typedef struct {
  int nx, ny, nz;
  double tau, kappa, beta, rho_l, rho_g, rho0;
  int scheme;
} o3_params;

typedef struct {
  double mass, umax, mu_min, mu_max, kinetic;
  int nonfinite;
} o3_stats;

static int wrap3(int a, int n) {
  if (a < 0) return a + n;
  if (a >= n) return a - n;
  return a;
}

static size_t node3(const o3_params* p, int x, int y, int z) {
  return ((size_t)wrap3(z, p->nz) * (size_t)p->ny + (size_t)wrap3(y, p->ny)) * (size_t)p->nx +
         (size_t)wrap3(x, p->nx);
}

/* Velocity set and weights, for tests that need to name a direction. */
void o3_lattice(int* cx, int* cy, int* cz, double* w) {
  for (int i = 0; i < Q3; ++i) {
    cx[i] = EX[i];
    cy[i] = EY[i];
    cz[i] = EZ[i];
    w[i] = WQ3(i);
  }
}

/* mu_0 = d psi_0 / d rho of psi_0 = beta (rho - rho_l)^2 (rho - rho_g)^2
 * (Eq. doubleWell), by the product rule. */
double o3_mu0(const o3_params* p, double rho) {
  double a = rho - p->rho_l, b = rho - p->rho_g;
  return 2.0 * p->beta * a * b * b + 2.0 * p->beta * a * a * b;
}

void o3_laplacian(const o3_params* p, const double* phi, double* out) {
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        double c = phi[node3(p, x, y, z)], s = 0.0;
        for (int i = 0; i < Q3; ++i)
          s += WQ3(i) * (phi[node3(p, x + EX[i], y + EY[i], z + EZ[i])] - c);
        out[node3(p, x, y, z)] = 2.0 / CS2_3 * s;
      }
}

void o3_gradient(const o3_params* p, const double* phi, double* gx, double* gy, double* gz) {
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int i = 0; i < Q3; ++i) {
          double v = phi[node3(p, x + EX[i], y + EY[i], z + EZ[i])];
          sx += WQ3(i) * EX[i] * v;
          sy += WQ3(i) * EY[i] * v;
          sz += WQ3(i) * EZ[i] * v;
        }
        size_t k = node3(p, x, y, z);
        gx[k] = sx / CS2_3;
        gy[k] = sy / CS2_3;
        gz[k] = sz / CS2_3;
      }
}

/* Equilibria: the standard one (Eq. feq) and the well-balanced one
 * (Eq. mFeq) at (rho, u). */
void o3_feq(const o3_params* p, double rho, const double* u, double* feq) {
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q3; ++i) {
    double cu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2];
    double P = cu / CS2_3 + cu * cu / (2.0 * CS2_3 * CS2_3) - uu / (2.0 * CS2_3);
    if (p->scheme == O3_WELL_BALANCED)
      feq[i] = i == 0 ? rho - (1.0 - WQ3(0)) * p->rho0 - WQ3(0) * rho * uu / (2.0 * CS2_3)
                      : WQ3(i) * (p->rho0 + rho * P);
    else
      feq[i] = WQ3(i) * rho * (1.0 + P);
  }
}

/* u A : (c_i c_i - cs^2 I), written out. */
static double contract3(int i, const double* u, const double* a) {
  const double c[D3] = {(double)EX[i], (double)EY[i], (double)EZ[i]};
  double s = 0.0;
  for (int al = 0; al < D3; ++al)
    for (int be = 0; be < D3; ++be)
      s += u[al] * a[be] * (c[al] * c[be] - (al == be ? CS2_3 : 0.0));
  return s;
}

/* Forcing terms: the standard Eq. Fi, or the well-balanced Eq. mFi with
 * D = 3 (G = F + cs^2 grad rho). */
void o3_forcing(const o3_params* p, const double* u, const double* F, const double* grho,
                double* Fi) {
  double G[D3], ugr = 0.0;
  for (int a = 0; a < D3; ++a) {
    G[a] = p->scheme == O3_WELL_BALANCED ? F[a] + CS2_3 * grho[a] : F[a];
    ugr += u[a] * grho[a];
  }
  for (int i = 0; i < Q3; ++i) {
    double cF = EX[i] * F[0] + EY[i] * F[1] + EZ[i] * F[2];
    double c2 = (double)(EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i]);
    double v = cF / CS2_3 + contract3(i, u, G) / (CS2_3 * CS2_3);
    if (p->scheme == O3_WELL_BALANCED) v += 0.5 * (c2 / CS2_3 - D3) * ugr;
    Fi[i] = WQ3(i) * v;
  }
}

/* rho, mu, u, F and grad(rho) of the state f (post-streaming); any output
 * pointer may be NULL.  Arrays of vectors are [3][n]. */
void o3_macro(const o3_params* p, const double* f, double* rho_out, double* mu_out,
              double* u_out, double* F_out, double* gr_out) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  double* rho = (double*)malloc(n * sizeof(double));
  double* lap = (double*)malloc(n * sizeof(double));
  double* mu = (double*)malloc(n * sizeof(double));
  double* gm = (double*)malloc(3 * n * sizeof(double));
  double* gr = (double*)malloc(3 * n * sizeof(double));
  for (size_t k = 0; k < n; ++k) {
#ifdef ORC_DENSITY_PAIRWISE
    double s = f[k];
    for (int i = 1; i < Q3; i += 2) s += f[(size_t)i * n + k] + f[(size_t)(i + 1) * n + k];
#else
    double s = 0.0;
    for (int i = 0; i < Q3; ++i) s += f[(size_t)i * n + k];
#endif
    rho[k] = s;
  }
  o3_laplacian(p, rho, lap);
  for (size_t k = 0; k < n; ++k) mu[k] = o3_mu0(p, rho[k]) - p->kappa * lap[k];
  o3_gradient(p, mu, gm, gm + n, gm + 2 * n);
  o3_gradient(p, rho, gr, gr + n, gr + 2 * n);
  for (size_t k = 0; k < n; ++k) {
    double F[D3], j[D3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D3; ++a)
      F[a] = p->scheme == O3_WELL_BALANCED ? -rho[k] * gm[a * n + k]
                                           : CS2_3 * gr[a * n + k] - rho[k] * gm[a * n + k];
    for (int i = 0; i < Q3; ++i) {
      j[0] += EX[i] * f[(size_t)i * n + k];
      j[1] += EY[i] * f[(size_t)i * n + k];
      j[2] += EZ[i] * f[(size_t)i * n + k];
    }
    if (rho_out) rho_out[k] = rho[k];
    if (mu_out) mu_out[k] = mu[k];
    for (int a = 0; a < D3; ++a) {
      if (u_out) u_out[a * n + k] = (j[a] + 0.5 * F[a]) / rho[k];
      if (F_out) F_out[a * n + k] = F[a];
      if (gr_out) gr_out[a * n + k] = gr[a * n + k];
    }
  }
  free(rho); free(lap); free(mu); free(gm); free(gr);
}

/* f = f^eq(rho, u = 0) (the runs start at rest, Sec. IV). */
void o3_init(const o3_params* p, const double* rho, double* f) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  const double zero[D3] = {0.0, 0.0, 0.0};
  double feq[Q3];
  for (size_t k = 0; k < n; ++k) {
    o3_feq(p, rho[k], zero, feq);
    for (int i = 0; i < Q3; ++i) f[(size_t)i * n + k] = feq[i];
  }
}

/* One step of Eq. D2Q9 on D3Q19: collision with the forcing term, then
 * streaming to x + c_i (periodic). */
static void o3_step_once(const o3_params* p, double* f, double* work) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  double* fnew = work;
  double* rho = work + (size_t)Q3 * n;
  double* u = rho + n;
  double* F = u + 3 * n;
  double* gr = F + 3 * n;
  double omega = 1.0 / p->tau, kforce = 1.0 - 1.0 / (2.0 * p->tau);
  o3_macro(p, f, rho, NULL, u, F, gr);
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        size_t k = node3(p, x, y, z);
        double uk[D3] = {u[k], u[n + k], u[2 * n + k]};
        double Fk[D3] = {F[k], F[n + k], F[2 * n + k]};
        double gk[D3] = {gr[k], gr[n + k], gr[2 * n + k]};
        double feq[Q3], Fi[Q3];
        o3_feq(p, rho[k], uk, feq);
        o3_forcing(p, uk, Fk, gk, Fi);
        for (int i = 0; i < Q3; ++i) {
          double fi = f[(size_t)i * n + k];
          double post = fi - omega * (fi - feq[i]) + kforce * Fi[i];
          fnew[(size_t)i * n + node3(p, x + EX[i], y + EY[i], z + EZ[i])] = post;
        }
      }
  memcpy(f, fnew, (size_t)Q3 * n * sizeof(double));
}

int o3_step(const o3_params* p, double* f, long nsteps) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  double* work = (double*)malloc((size_t)(Q3 + 10) * n * sizeof(double));
  if (!work) return -1;
  for (long s = 0; s < nsteps; ++s) o3_step_once(p, f, work);
  free(work);
  return 0;
}

/* mass (compensated sum), max |u|, min/max mu, E = 1/2 sum rho |u|^2 and a
 * flag for any non-finite value (Sec. IV). */
void o3_stats_of(const o3_params* p, const double* f, o3_stats* st) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  double* rho = (double*)malloc(n * sizeof(double));
  double* mu = (double*)malloc(n * sizeof(double));
  double* u = (double*)malloc(3 * n * sizeof(double));
  o3_macro(p, f, rho, mu, u, NULL, NULL);
  double sum = 0.0, comp = 0.0, umax = 0.0, e = 0.0, mumin = INFINITY, mumax = -INFINITY;
  int bad = 0;
  for (size_t k = 0; k < n; ++k) {
    double yk = rho[k] - comp, t = sum + yk;
    comp = (t - sum) - yk;
    sum = t;
    double u2 = u[k] * u[k] + u[n + k] * u[n + k] + u[2 * n + k] * u[2 * n + k];
    if (sqrt(u2) > umax) umax = sqrt(u2);
    if (mu[k] < mumin) mumin = mu[k];
    if (mu[k] > mumax) mumax = mu[k];
    e += 0.5 * rho[k] * u2;
    if (!isfinite(rho[k]) || !isfinite(mu[k]) || !isfinite(u2)) bad = 1;
  }
  st->mass = sum;
  st->umax = umax;
  st->mu_min = mumin;
  st->mu_max = mumax;
  st->kinetic = e;
  st->nonfinite = bad;
  free(rho); free(mu); free(u);
}
