// Fused collide-stream kernels for the standard (Sec. II) and well-balanced
// (Sec. III) D2Q9 LBE of Guo, arXiv 2012.11075, written for sm_103a.
//
// State layout: nine structure-of-arrays planes P_i[y * pitch + x] holding
// the post-collision populations of the previous step, so that the
// pre-collision populations of step t are pulled as
//     f_i(x, t) = P_i(x - c_i)                          (streaming, Eq. D2Q9)
// with periodic wrap.  In FP32-shifted storage the planes hold
// g_i = f_i - s_i (see wblbe.h); in FP64 they hold f_i.
//
// One CTA owns a strip of tile_x lattice columns and marches a run of rows
// upward.  For every row it stages the nine plane rows its columns pull from
// (plus four halo columns on each side) in shared memory with asynchronous
// copies issued several rows ahead of use, reduces them to the density
// (Eq. rhoU) and keeps the densities of the last rows in a shared-memory
// ring.  The chemical potential
// mu = mu_0(rho) - kappa lap(rho) of the row below is computed into a second
// ring, and the row two below the load front is collided: gradients of mu
// and rho (isotropic central stencil), the interaction force (Eq. mF, or a
// force form of Sec. II), the velocity (Eq. rhoU), the equilibrium and
// forcing terms (Eq. mFeq/mFi or Eq. feq/Fi) and the BGK update are all
// evaluated in registers, and the nine results are stored to the other
// buffer.  Each population is read from DRAM once per step (the halo rows and
// columns of neighbouring strips come from L2), and written once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wblbe {

constexpr int kHalo = 2;          // density halo radius (mu needs 1, grad mu 2)
constexpr int kMaxTile = 256;

// Parameters of one launch, passed by value.
struct KParams {
  int nx, ny, pitch, rows;        // rows: lattice rows marched by one CTA
  long long plane;                // elements per population plane
  // physics (stored as double; cast to the arithmetic type in the kernel)
  double omega;                   // 1/tau
  double kforce;                  // 1 - 1/(2 tau)
  double kappa;
  double two_beta;                // 2 beta
  double dl, dg;                  // rho_ref - rho_l, rho_ref - rho_g
  double rho_ref;                 // 0 in FP64
  // Time step t of the state being updated, which seeds the stochastic
  // rounding of the FP32 well-balanced update: t = step + *step_base
  // (step_base may be null; a graph replay reads its base from device memory).
  long long step;
  const long long* step_base;
  // Rows of the stored lattice a step or moments launch updates, [row_lo,
  // row_hi) (the whole lattice: 0, ny), and the offset from a stored row to
  // its row in the global lattice (0, except for a slab of a lattice split
  // into row slabs: there the stored rows are the slab's rows and the ghost
  // rows around them).
  int row_lo, row_hi, y_offset;
};

// Outputs of the moments mode (any pointer may be null).
struct MomentsOut {
  double* rho;
  double* ux;
  double* uy;
  double* mu;
  double* partials;               // per-CTA stats records (kStatRec doubles)
};

constexpr int kStatRec = 6;       // mass, kinetic, umax^2, mu_min, mu_max, nonfinite

// Schemes (the values of the C ABI's scheme codes): the standard LBE of
// Sec. II (potential-form force, Eq. Fi), the well-balanced LBE of Sec. III,
// and two variants of the standard LBE that Sec. II compares: the
// pressure-form force grad(cs^2 rho - p_0) + kappa rho grad(lap rho), and the
// forcing term F_i = (c_i - u).F f_i^eq / (cs^2 rho) of Guo's textbook.
enum SchemeId : int { kSchStandard = 0, kSchWB = 1, kSchPressure = 2, kSchTextbook = 3 };

// Bounds-checked build (-DWBLBE_DEBUG_BOUNDS): every global access of the
// strip kernels and the shared-memory slots computed at run time are checked
// before use; a bad access is skipped and counted in g_bounds_errors (no
// trap), which the host reads with wblbe_debug_bounds_errors.  Without the
// flag the checks compile to nothing.
#ifdef WBLBE_DEBUG_BOUNDS
static __device__ unsigned int g_bounds_errors;
__device__ __forceinline__ bool in_bounds(long long off, long long n) {
  if (off >= 0 && off < n) return true;
  atomicAdd(&g_bounds_errors, 1u);
  return false;
}
// host side, per translation unit: read (and optionally clear) the count
static unsigned int read_bounds_errors(bool reset) {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_errors, sizeof(v)) != cudaSuccess) return 0xFFFFFFFEu;
  if (reset) {
    const unsigned int z = 0;
    cudaMemcpyToSymbol(g_bounds_errors, &z, sizeof(z));
  }
  return v;
}
#define WB_IN(off, n) ::wblbe::in_bounds((long long)(off), (long long)(n))
#else
static inline unsigned int read_bounds_errors(bool) { return 0xFFFFFFFFu; }
#define WB_IN(off, n) true
#endif

__device__ __forceinline__ int wrap_index(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// mu = mu_0(rho) - kappa lap(rho) at one node from the 3x3 neighbourhood of
// stored densities rs (rho = rs + rho_ref):
//   mu_0 = 2 beta (rho - rho_l)(rho - rho_g)(2 rho - rho_l - rho_g)
//   lap  = [4 (E + W + N + S) + (NE + NW + SE + SW) - 20 C] / 6
// kappa6 = kappa / 6.
template <typename T>
__device__ __forceinline__ T chem_pot(T c, T e, T w, T n, T s, T ne, T nw, T se,
                                      T sw, T two_beta, T dl, T dg, T kappa6) {
  T a = c + dl, b = c + dg;
  T mu0 = two_beta * a * b * (a + b);
  T lap6 = T(4) * ((e + w) + (n + s)) + ((ne + nw) + (se + sw)) - T(20) * c;
  return mu0 - kappa6 * lap6;
}

// chem_pot with the row sums ew = e + w, nenw = ne + nw and sesw = se + sw
// passed in (the FP64 strip kernel forms each row's sum once and carries it
// to the two rows above): the same operations in the same order, so the
// same result.
template <typename T>
__device__ __forceinline__ T chem_pot_rows(T c, T ew, T n, T s, T nenw, T sesw, T two_beta,
                                           T dl, T dg, T kappa6) {
  T a = c + dl, b = c + dg;
  T mu0 = two_beta * a * b * (a + b);
  T lap6 = T(4) * (ew + (n + s)) + (nenw + sesw) - T(20) * c;
  return mu0 - kappa6 * lap6;
}

// 1/x: the hardware reciprocal approximation in FP32 (about 1 ulp; the FP32
// path's error budget is set by float storage anyway).
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The hardware's FP64 reciprocal approximation (rcp.approx.ftz.f64), the
// seed of recip(double).
__device__ __forceinline__ double recip_seed(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

// 1/x in FP64 for the density (normal, positive in any valid state): the
// hardware seed r, then one step of the third-order Householder iteration
// for the reciprocal, r <- r + r (e + e^2) with e = 1 - x r (two fused
// multiply-adds and one more for the update), which cubes the seed's
// relative error.  Three FP64 instructions after the seed, where the IEEE
// division takes several more and a slow-path test; its accuracy against
// the IEEE quotient is checked on the GPU (wblbe_probe_reciprocal).  A zero
// or non-finite x gives a non-finite result.
__device__ __forceinline__ double recip(double x) {
  const double r = recip_seed(x);
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// Collision constants in the arithmetic type, converted once per kernel (a
// float <- double conversion inside the row loop would run on the FP64 pipe).
// The rho0 terms of the well-balanced equilibrium never reach the kernel: in
// both precisions the planes store deviations from a shift that contains the
// node-independent rho0 vector (-(1-w0) rho0, w_i rho0), which the BGK update
// and streaming carry unchanged.
// keep = 1 - omega must hold exactly in the arithmetic type: the update
// keep * g + omega * (...) conserves mass only if keep + omega == 1, and a
// rounded pair would scale the mass every step.  For omega >= 1/2 (tau <= 2)
// 1 - omega is exact (Sterbenz); for smaller omega, omega is taken as 1 - keep.
template <typename T>
struct CollideConsts {
  T omega, kf, keep, kf_m3, rho_ref, kappa, kf12;
  T kfm12, kf36, kf432;             // -kforce/12, kforce/36, kforce/432 (collide_wb12)
  __device__ explicit CollideConsts(const KParams& p)
      : kf(T(p.kforce)), kf_m3(T(-3.0 * p.kforce)), rho_ref(T(p.rho_ref)), kappa(T(p.kappa)),
        kf12(T(p.kforce / 12.0)), kfm12(T(-p.kforce / 12.0)), kf36(T(p.kforce / 36.0)),
        kf432(T(p.kforce / 432.0)) {
    const T w = T(p.omega);
    if (w >= T(0.5)) {
      omega = w;
      keep = T(1) - w;
    } else {
      keep = T(1.0 - p.omega);
      omega = T(1) - keep;
    }
  }
};

// Collision of one node in stored variables.  Inputs: the nine pulled
// populations g, the stored density rs (rho = rs + rho_ref), gradients of mu
// and rho.  Outputs: the nine post-collision stored populations (into g) and
// the velocity.
//
// With w_i, P_i = 3 c.u + 9/2 (c.u)^2 - 3/2 u.u and the base terms b_i
// (FP64: the rest equilibrium; FP32-shifted: its deviation from s_i) every
// equilibrium of both schemes is b_i + w_i rho P_i, and the forcing terms are
//   F_i = w_i [3 c.F + 9 (c.u)(c.G) - 3 u.G + h_i (u.grad rho)]
// with G = F + cs^2 grad rho, h_i = (3|c_i|^2 - 2)/2 for the well-balanced
// scheme (Eq. mFi) and G = F, h_i = 0 for the standard one (Eq. Fi).  Each
// pair of opposite directions shares the even part E and flips the odd
// part O of  omega feq_i + kforce F_i.  With t = omega rho (-3/2 u.u) +
// kforce (-3 u.G) and k_u = kforce (u.grad rho):
//   E_0 = w_0 (t - k_u) + omega b_0,   E_axis base = w_ax (t + k_u/2) + omega b_ax,
//   E_diag base = w_dg (t + 2 k_u) + omega b_dg.
// The variants of the standard scheme: with the pressure form the gradient
// inputs are grad(lap rho) (gm) and grad(cs^2 rho - p_0) (gr); with the
// textbook forcing term the collision takes textbook_pairs below.
template <typename T>
__device__ __forceinline__ void textbook_pairs(T (&g)[9], T rs, T rho, T ux, T uy, T Fx,
                                               T Fy, const CollideConsts<T>& q);

// The well-balanced collision from 12 grad mu and 12 grad rho (iso_grad12),
// the same terms as collide below arranged for fewer operations, which is
// what bounds the FP64 path.  F = -rho grad mu enters the update only as F/2
// (the velocity, Eq. rhoU) and as kforce F, so both are formed from the
// gradient directly; G = F + cs^2 grad rho enters only as kforce G; and t,
// k_u are carried divided by 36, so that the even parts are
// E_dg = t' + 2 k_u', E_ax = 3 t' + E_dg and E_0 = 16 (t' - k_u') + omega b_0.
template <typename T>
__device__ __forceinline__ void collide_wb12(T (&g)[9], T rs, T gmx, T gmy, T grx, T gry,
                                             const CollideConsts<T>& q, T& ux_out,
                                             T& uy_out) {
  constexpr bool kShifted = sizeof(T) == 4;
  const T omega = q.omega;
  const T rho = kShifted ? rs + q.rho_ref : rs;
  const T hm = rho * T(-1.0 / 24.0);                   // F/2 = hm (12 grad mu)
  const T kcm = rho * q.kfm12;                         // kforce F = kcm (12 grad mu)
  const T d13 = g[1] - g[3], d24 = g[2] - g[4], d57 = g[5] - g[7], d86 = g[8] - g[6];
  const T jx = (d13 + d57) + d86;
  const T jy = (d24 + d57) - d86;
  const T inv_rho = recip(rho);
  const T ux = (jx + hm * gmx) * inv_rho;               // Eq. rhoU
  const T uy = (jy + hm * gmy) * inv_rho;
  ux_out = ux;
  uy_out = uy;
  const T kFx = kcm * gmx, kFy = kcm * gmy;
  const T kGx = kFx + q.kf36 * grx, kGy = kFy + q.kf36 * gry;
  const T orho = omega * rho;
  const T uu = ux * ux + uy * uy;
  const T uK = ux * kGx + uy * kGy;                     // kforce u.G
  const T tq = (orho * T(-1.0 / 24.0)) * uu - T(1.0 / 12.0) * uK;   // t / 36
  const T kq = q.kf432 * (ux * grx + uy * gry);         // k_u / 36
  const T Cdg = tq + T(2) * kq;
  const T Cax = T(3) * tq + Cdg;
  const T E0 = T(16) * (tq - kq) + omega * rs;          // b_0 = rs, b_ax = b_dg = 0
  const T hrho = T(0.5) * orho;
  const T Mx = orho * ux + kFx;                         // odd parts: omega rho c.u + kforce c.F
  const T My = orho * uy + kFy;
  const T E1 = Cax + ux * (hrho * ux + kGx);            // pair (1,3): c = (1,0)
  const T O1 = T(1.0 / 3.0) * Mx;
  const T E2 = Cax + uy * (hrho * uy + kGy);            // pair (2,4): c = (0,1)
  const T O2 = T(1.0 / 3.0) * My;
  const T cu5 = ux + uy;                                // pair (5,7): c = (1,1)
  const T E5 = Cdg + (T(0.25) * cu5) * (hrho * cu5 + (kGx + kGy));
  const T O5 = T(1.0 / 12.0) * (Mx + My);
  const T cu6 = uy - ux;                                // pair (6,8): c = (-1,1)
  const T E6 = Cdg + (T(0.25) * cu6) * (hrho * cu6 + (kGy - kGx));
  const T O6 = T(1.0 / 12.0) * (My - Mx);
  const T keep = q.keep;
  g[1] = keep * g[1] + (E1 + O1);
  g[3] = keep * g[3] + (E1 - O1);
  g[2] = keep * g[2] + (E2 + O2);
  g[4] = keep * g[4] + (E2 - O2);
  g[5] = keep * g[5] + (E5 + O5);
  g[7] = keep * g[7] + (E5 - O5);
  g[6] = keep * g[6] + (E6 + O6);
  g[8] = keep * g[8] + (E6 - O6);
  if (kShifted) {
    (void)E0;                                           // mass balance, as in collide
    g[0] = rs - (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])));
  } else {
    g[0] = keep * g[0] + E0;
  }
}

// GS: the gradient inputs are GS times the gradients (12: the strip kernel
// passes 12 grad, see iso_grad12, and the factor 1/12 is folded into the
// few places that use them; 1: plain gradients).
template <typename T, int SCH, int GS = 1>
__device__ __forceinline__ void collide(T (&g)[9], T rs, T gmx, T gmy, T grx,
                                        T gry, const CollideConsts<T>& q, T& ux_out,
                                        T& uy_out) {
  constexpr bool WB = SCH == kSchWB;
  constexpr bool kShifted = sizeof(T) == 4;   // FP32 storage is always shifted
  constexpr bool kG12 = GS == 12;
  static_assert(GS == 1 || GS == 12, "gradient scale");
  if constexpr (WB && kG12) {
    collide_wb12<T>(g, rs, gmx, gmy, grx, gry, q, ux_out, uy_out);
    return;
  }
  const T omega = q.omega, kf = q.kf;
  // FP64 storage is unshifted (rho_ref = 0)
  const T rho = kShifted ? rs + q.rho_ref : rs;
  T Fx, Fy;
  if (kG12) {
    const T nr = rho * T(-1.0 / 12.0);                   // -rho / 12
    if (WB) {
      Fx = nr * gmx;                                     // Eq. mF
      Fy = nr * gmy;
    } else if (SCH == kSchPressure) {
      const T kr = q.kappa * rho;                        // pressure form
      Fx = T(1.0 / 12.0) * (grx + kr * gmx);
      Fy = T(1.0 / 12.0) * (gry + kr * gmy);
    } else {
      Fx = T(1.0 / 36.0) * grx + nr * gmx;               // potential form
      Fy = T(1.0 / 36.0) * gry + nr * gmy;
    }
  } else if (WB) {
    Fx = -rho * gmx;                                     // Eq. mF
    Fy = -rho * gmy;
  } else if (SCH == kSchPressure) {
    Fx = grx + q.kappa * rho * gmx;                      // pressure form
    Fy = gry + q.kappa * rho * gmy;
  } else {
    Fx = T(1.0 / 3.0) * grx - rho * gmx;                 // potential form
    Fy = T(1.0 / 3.0) * gry - rho * gmy;
  }
  const T d13 = g[1] - g[3], d24 = g[2] - g[4], d57 = g[5] - g[7], d86 = g[8] - g[6];
  const T jx = (d13 + d57) + d86;
  const T jy = (d24 + d57) - d86;
  const T inv_rho = recip(rho);
  const T ux = (jx + T(0.5) * Fx) * inv_rho;            // Eq. rhoU
  const T uy = (jy + T(0.5) * Fy) * inv_rho;
  ux_out = ux;
  uy_out = uy;
  if (SCH == kSchTextbook) {
    textbook_pairs<T>(g, rs, rho, ux, uy, Fx, Fy, q);
    return;
  }

  T Gx = Fx, Gy = Fy;
  if (WB) {
    Gx = Fx + T(kG12 ? 1.0 / 36.0 : 1.0 / 3.0) * grx;
    Gy = Fy + T(kG12 ? 1.0 / 36.0 : 1.0 / 3.0) * gry;
  }
  const T orho = omega * rho;
  const T uu = ux * ux + uy * uy;
  const T uG = ux * Gx + uy * Gy;
  const T t = (T(-1.5) * orho) * uu + q.kf_m3 * uG;

  T E0, Cax, Cdg;
  if (WB) {
    const T ku = (kG12 ? q.kf12 : kf) * (ux * grx + uy * gry);
    E0 = T(4.0 / 9.0) * (t - ku);
    Cax = T(1.0 / 9.0) * (t + T(0.5) * ku);
    Cdg = T(1.0 / 36.0) * (t + T(2) * ku);
    E0 = E0 + omega * rs;                              // b_0 = rs, b_ax = b_dg = 0
  } else {
    const T s = t + omega * rs;                        // b_i = w_i rs
    E0 = T(4.0 / 9.0) * s;
    Cax = T(1.0 / 9.0) * s;
    Cdg = T(1.0 / 36.0) * s;
  }
  const T hrho = T(0.5) * orho;              // (omega rho / 9) * 9/2
  const T kGx = kf * Gx, kGy = kf * Gy;
  const T Mx = orho * ux + kf * Fx;          // odd parts: omega rho c.u + kf c.F
  const T My = orho * uy + kf * Fy;

  // pair (1,3): c = (1,0)
  const T E1 = Cax + ux * (hrho * ux + kGx);
  const T O1 = T(1.0 / 3.0) * Mx;
  // pair (2,4): c = (0,1)
  const T E2 = Cax + uy * (hrho * uy + kGy);
  const T O2 = T(1.0 / 3.0) * My;
  // pair (5,7): c = (1,1)
  const T cu5 = ux + uy;
  const T E5 = Cdg + (T(0.25) * cu5) * (hrho * cu5 + (kGx + kGy));
  const T O5 = T(1.0 / 12.0) * (Mx + My);
  // pair (6,8): c = (-1,1)
  const T cu6 = uy - ux;
  const T E6 = Cdg + (T(0.25) * cu6) * (hrho * cu6 + (kGy - kGx));
  const T O6 = T(1.0 / 12.0) * (My - Mx);

  const T keep = q.keep;
  g[1] = keep * g[1] + (E1 + O1);
  g[3] = keep * g[3] + (E1 - O1);
  g[2] = keep * g[2] + (E2 + O2);
  g[4] = keep * g[4] + (E2 - O2);
  g[5] = keep * g[5] + (E5 + O5);
  g[7] = keep * g[7] + (E5 - O5);
  g[6] = keep * g[6] + (E6 + O6);
  g[8] = keep * g[8] + (E6 - O6);
  if (kShifted) {
    // The collision conserves the node's mass: sum_i g_i' = rs (exactly, in
    // real arithmetic).  In float storage the rest population g_0 ~ rho -
    // rho_ref is large, and the small one-signed O(u^2) part of E0 would be
    // lost to rounding when added to it, while the matching corrections to
    // the small moving populations survive: a systematic mass gain.  Taking
    // g_0' from the mass balance leaves only unbiased rounding.
    (void)E0;
    g[0] = rs - (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])));
  } else {
    g[0] = keep * g[0] + E0;
  }
}

// BGK update with the textbook forcing term F_i = (c_i - u).F f_i^eq /
// (cs^2 rho) = 3 w_i (1 + P_i)(c_i.F - u.F), standard equilibrium
// f_i^eq - s_i = w_i (rs + rho P_i).  For a pair (i, opposite) with
// e = 1 + 9/2 (c.u)^2 - 3/2 u.u (the even part of 1 + P_i) the even and odd
// parts of omega (f^eq - s) + kforce F are
//   E = omega w (rs + rho (e - 1)) + kforce 3w (3 (c.u)(c.F) - e u.F),
//   O = omega w rho 3 c.u + kforce 3w (e c.F - 3 (c.u) u.F).
template <typename T>
__device__ __forceinline__ void textbook_pairs(T (&g)[9], T rs, T rho, T ux, T uy, T Fx,
                                               T Fy, const CollideConsts<T>& q) {
  constexpr bool kShifted = sizeof(T) == 4;
  const T omega = q.omega, kf = q.kf, keep = q.keep;
  const T uu = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
  const T e0 = T(1) - T(1.5) * uu;
  auto pair = [&](T w, T cu, T cF, T& E, T& O) {
    const T e = e0 + T(4.5) * cu * cu;
    E = omega * w * (rs + rho * (e - T(1))) + kf * T(3) * w * (T(3) * cu * cF - e * uF);
    O = omega * w * rho * T(3) * cu + kf * T(3) * w * (e * cF - T(3) * cu * uF);
  };
  T E, O;
  pair(T(1.0 / 9.0), ux, Fx, E, O);
  g[1] = keep * g[1] + (E + O);
  g[3] = keep * g[3] + (E - O);
  pair(T(1.0 / 9.0), uy, Fy, E, O);
  g[2] = keep * g[2] + (E + O);
  g[4] = keep * g[4] + (E - O);
  pair(T(1.0 / 36.0), ux + uy, Fx + Fy, E, O);
  g[5] = keep * g[5] + (E + O);
  g[7] = keep * g[7] + (E - O);
  pair(T(1.0 / 36.0), uy - ux, Fy - Fx, E, O);
  g[6] = keep * g[6] + (E + O);
  g[8] = keep * g[8] + (E - O);
  if (kShifted) {
    g[0] = rs - (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])));
  } else {
    const T w0 = T(4.0 / 9.0);
    g[0] = keep * g[0] + (omega * w0 * (rs + rho * (e0 - T(1))) - kf * T(3) * w0 * e0 * uF);
  }
}

// Isotropic central gradient from the 3x3 neighbourhood:
//   grad_x = (E - W)/3 + (NE + SE - NW - SW)/12,
//   grad_y = (N - S)/3 + (NE + NW - SE - SW)/12,
// written with the diagonal differences d1 = NE - SW, d2 = SE - NW.
template <typename T>
__device__ __forceinline__ void iso_grad(T e, T w, T n, T s, T ne, T nw, T se, T sw,
                                         T& gx, T& gy) {
  const T d1 = ne - sw, d2 = se - nw;
  gx = T(1.0 / 3.0) * (e - w) + T(1.0 / 12.0) * (d1 + d2);
  gy = T(1.0 / 3.0) * (n - s) + T(1.0 / 12.0) * (d1 - d2);
}

// 12 times the same gradient, 4 (E - W) + (d1 + d2): two multiplications
// fewer per gradient; collide<T, SCH, 12> folds the 1/12 into its uses.
template <typename T>
__device__ __forceinline__ void iso_grad12(T e, T w, T n, T s, T ne, T nw, T se, T sw,
                                           T& gx, T& gy) {
  const T d1 = ne - sw, d2 = se - nw;
  gx = T(4) * (e - w) + (d1 + d2);
  gy = T(4) * (n - s) + (d1 - d2);
}

// iso_grad12 from per-row x-differences q = f(x+1) - f(x-1) and x-sums
// p = f(x+1) + f(x-1) of the rows above (n), at (c) and below (s), which
// the FP64 strip kernel forms once per row and carries:
// 12 df/dx = 4 q_c + (q_n + q_s),  12 df/dy = 4 (n - s) + (p_n - p_s).
template <typename T>
__device__ __forceinline__ void iso_grad12_rows(T qc, T qn, T qs, T n, T s, T pn, T ps, T& gx,
                                                T& gy) {
  gx = T(4) * qc + (qn + qs);
  gy = T(4) * (n - s) + (pn - ps);
}

// ---- packed FP32 pairs ------------------------------------------------------
//
// In FP32 a thread advances two lattice rows per iteration; their arithmetic
// is identical, so it runs on float2 pairs (x: the lower row, y: the upper
// row) with the paired FP32 instructions of sm_100 and later, one instruction
// for both rows.  Each lane is an ordinary IEEE single-precision operation,
// so a row's result does not depend on which lane it occupies.
__device__ __forceinline__ float2 splat(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ---- exact-mass rest population of the FP32 well-balanced update -----------
//
// The collision conserves each node's mass exactly in real arithmetic
// (sum_i f^eq_i = rho and sum_i F_i = 0, Sec. III), so the post-collision
// rest population is g_0' = g_0 + (m - a), m and a the sums of the pulled
// and of the post-collision moving populations.  In float storage the rest
// population (about rho - rho_ref) is much larger than the moving ones
// (O(u, F) in the well-balanced scheme), so the roundings that enter m - a
// (the moving populations' own, and those of the sums) are far below an
// ulp of g_0, and one error-free addition (TwoSum) gives
// g_0 + (m - a) = h + e exactly.  g_0' is h or its float neighbour on the
// side of e, the neighbour with probability |e| / (distance to it): the
// expected rounding error is zero, so a state that repeats its rounding step
// after step (near equilibrium) no longer drifts in mass; its mass performs
// a random walk instead.  The random bits come from a counter-based hash of
// the node (x, y) and the time step t, so results do not depend on the
// launch shape, on batching or on the order in which tiles run.

// Error-free sum (Knuth's TwoSum) on a pair of lanes: s = fl(a + b) and
// a + b = s + e exactly.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bv = sub2(s, a);
  e = add2(sub2(a, sub2(s, bv)), sub2(b, bv));
}

// MurmurHash3's 32-bit finalizer (Appleby): a bijective avalanche mixer.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Key of time step t (folded into every node's hash of that step).
__device__ __forceinline__ uint32_t step_key(long long t) {
  return fmix32((uint32_t)t * 0x9e3779b9u + 0x6a09e667u);
}

// Uniform draws in [0, 1) on a 2^-23 grid for the two nodes of column x in
// rows 2j and 2j + 1 (k = 2j nx + x is the lower node's key): one hash of k
// and the step key ht; the upper node's draw takes the top bits of the hash
// times an odd constant, which every bit of the hash feeds.  The pairing is
// by absolute row, so a node's draw does not depend on the launch shape.
__device__ __forceinline__ float2 pair_uniforms(uint32_t k, uint32_t ht) {
  const uint32_t h = fmix32(k + ht);
  const uint32_t h2 = h * 0x9e3779b9u;
  // 1.m - 1 with the 23 random bits as the mantissa m: exact
  return make_float2(__fsub_rn(__uint_as_float(0x3f800000u | (h >> 9)), 1.0f),
                     __fsub_rn(__uint_as_float(0x3f800000u | (h2 >> 9)), 1.0f));
}

// The float next to h on the side of e: one step of the bit pattern away
// from zero when e and h have the same sign bit, towards zero otherwise.
// For a zero h it is a NaN or the smallest subnormal, for the largest finite
// h an infinity (round_stochastic2 then keeps h or rounds to that tiny value).
__device__ __forceinline__ float next_toward(float h, float e) {
  const int b = __float_as_int(h);
  const int s = (__float_as_int(e) ^ b) >> 31;        // 0: same sign, -1: opposite
  return __int_as_float(b + 1 + 2 * s);
}

// Round v = h + e on a pair of lanes (e the exact remainder, |e| at most
// half an ulp of h) to h or to the float next to h on the side of e,
// choosing the neighbour with probability |e| / gap (gap = the exact
// distance to it, a power of two); u uniform in [0, 1) on a 2^-23 grid.
// E[result] = v up to 2^-23 of a gap.  An infinite or NaN h is kept.
__device__ __forceinline__ float2 round_stochastic2(float2 h, float2 e, float2 u) {
  const float2 n = make_float2(next_toward(h.x, e.x), next_toward(h.y, e.y));
  const float2 ug = mul2(u, sub2(n, h));               // u times the signed gap
  return make_float2(fabsf(ug.x) < fabsf(e.x) ? n.x : h.x, fabsf(ug.y) < fabsf(e.y) ? n.y : h.y);
}

// Mirror-symmetric sum of the eight moving populations: every lattice
// mirror (x, y, diagonal) maps the grouping onto itself, so mirror-image
// nodes round alike and the rounding leaves no net force.
__device__ __forceinline__ float2 moving_sum2(const float2 (&g)[9]) {
  return add2(add2(add2(g[1], g[3]), add2(g[2], g[4])), add2(add2(g[5], g[7]), add2(g[6], g[8])));
}

// chem_pot on a pair of nodes (same formula and evaluation order)
__device__ __forceinline__ float2 chem_pot_x2(float2 c, float2 e, float2 w, float2 n, float2 s,
                                              float2 ne, float2 nw, float2 se, float2 sw,
                                              float2 two_beta, float2 dl, float2 dg,
                                              float2 kappa6) {
  const float2 a = add2(c, dl), b = add2(c, dg);
  const float2 mu0 = mul2(mul2(mul2(two_beta, a), b), add2(a, b));
  const float2 lap6 = fma2(splat(-20.0f), c,
                           fma2(splat(4.0f), add2(add2(e, w), add2(n, s)),
                                add2(add2(ne, nw), add2(se, sw))));
  return fma2(kappa6, make_float2(-lap6.x, -lap6.y), mu0);
}

// iso_grad on a pair of nodes
__device__ __forceinline__ void iso_grad_x2(float2 e, float2 w, float2 n, float2 s, float2 ne,
                                            float2 nw, float2 se, float2 sw, float2& gx,
                                            float2& gy) {
  const float2 d1 = sub2(ne, sw), d2 = sub2(se, nw);
  gx = fma2(splat(1.0f / 3.0f), sub2(e, w), mul2(splat(1.0f / 12.0f), add2(d1, d2)));
  gy = fma2(splat(1.0f / 3.0f), sub2(n, s), mul2(splat(1.0f / 12.0f), sub2(d1, d2)));
}

// textbook_pairs<float> on a pair of nodes
__device__ __forceinline__ void textbook_pairs_x2(float2 (&g)[9], float2 rs, float2 rho,
                                                  float2 ux, float2 uy, float2 Fx, float2 Fy,
                                                  const CollideConsts<float>& q) {
  const float2 omega = splat(q.omega), kf3 = mul2(splat(q.kf), splat(3.0f)), keep = splat(q.keep);
  const float2 uu = fma2(ux, ux, mul2(uy, uy)), uF = fma2(ux, Fx, mul2(uy, Fy));
  const float2 e0 = fma2(splat(-1.5f), uu, splat(1.0f));
  const float2 orho = mul2(omega, rho);
  auto pair = [&](float w, float2 cu, float2 cF, float2& E, float2& O) {
    const float2 e = fma2(mul2(splat(4.5f), cu), cu, e0);
    const float2 em1 = sub2(e, splat(1.0f));
    const float2 fe = mul2(splat(w), fma2(rho, em1, rs));
    const float2 fo = mul2(splat(3.0f * w), mul2(orho, cu));
    const float2 t3 = mul2(splat(3.0f), cu);
    E = fma2(omega, fe, mul2(mul2(kf3, splat(w)), sub2(mul2(t3, cF), mul2(e, uF))));
    O = fma2(mul2(kf3, splat(w)), sub2(mul2(e, cF), mul2(t3, uF)), fo);
  };
  float2 E, O;
  pair(1.0f / 9.0f, ux, Fx, E, O);
  g[1] = fma2(keep, g[1], add2(E, O));
  g[3] = fma2(keep, g[3], sub2(E, O));
  pair(1.0f / 9.0f, uy, Fy, E, O);
  g[2] = fma2(keep, g[2], add2(E, O));
  g[4] = fma2(keep, g[4], sub2(E, O));
  pair(1.0f / 36.0f, add2(ux, uy), add2(Fx, Fy), E, O);
  g[5] = fma2(keep, g[5], add2(E, O));
  g[7] = fma2(keep, g[7], sub2(E, O));
  pair(1.0f / 36.0f, sub2(uy, ux), sub2(Fy, Fx), E, O);
  g[6] = fma2(keep, g[6], add2(E, O));
  g[8] = fma2(keep, g[8], sub2(E, O));
  g[0] = sub2(rs, add2(add2(add2(g[1], g[3]), add2(g[2], g[4])),
                       add2(add2(g[5], g[7]), add2(g[6], g[8]))));
}

// collide<float, SCH> on a pair of nodes (FP32-shifted storage): the same
// terms as the scalar version, with the multiply-adds written out.
// rnd: a uniform draw per lane for the stochastic rounding of the rest
// population (well-balanced scheme only, see round_stochastic).
template <int SCH>
__device__ __forceinline__ void collide_x2(float2 (&g)[9], float2 rs, float2 gmx, float2 gmy,
                                           float2 grx, float2 gry, const CollideConsts<float>& q,
                                           float2& ux_out, float2& uy_out, float2 rnd) {
  constexpr bool WB = SCH == kSchWB;
  const float2 omega = splat(q.omega), kf = splat(q.kf), third = splat(1.0f / 3.0f);
  const float2 rho = add2(rs, splat(q.rho_ref));
  const float2 nrho = sub2(splat(-q.rho_ref), rs);        // -rho
  float2 Fx, Fy;
  if (WB) {
    Fx = mul2(nrho, gmx);                                 // Eq. mF
    Fy = mul2(nrho, gmy);
  } else if (SCH == kSchPressure) {
    const float2 krho = mul2(splat(q.kappa), rho);        // pressure form
    Fx = fma2(krho, gmx, grx);
    Fy = fma2(krho, gmy, gry);
  } else {
    Fx = fma2(third, grx, mul2(nrho, gmx));               // potential form
    Fy = fma2(third, gry, mul2(nrho, gmy));
  }
  const float2 d13 = sub2(g[1], g[3]), d24 = sub2(g[2], g[4]);
  const float2 d57 = sub2(g[5], g[7]), d86 = sub2(g[8], g[6]);
  // mirror-symmetric groupings: an x-mirror negates jx exactly, a y-mirror jy
  const float2 jx = add2(d13, add2(d57, d86));
  const float2 jy = add2(d24, sub2(d57, d86));
  // pulled moving populations' sum (rs is g_0 plus this, formed in staging)
  const float2 m_in = WB ? moving_sum2(g) : make_float2(0.f, 0.f);
  const float2 inv_rho = make_float2(recip(rho.x), recip(rho.y));
  const float2 half = splat(0.5f);
  const float2 ux = mul2(fma2(half, Fx, jx), inv_rho);   // Eq. rhoU
  const float2 uy = mul2(fma2(half, Fy, jy), inv_rho);
  ux_out = ux;
  uy_out = uy;
  if (SCH == kSchTextbook) {
    textbook_pairs_x2(g, rs, rho, ux, uy, Fx, Fy, q);
    return;
  }

  float2 Gx = Fx, Gy = Fy;
  if (WB) {
    Gx = fma2(third, grx, Fx);
    Gy = fma2(third, gry, Fy);
  }
  const float2 orho = mul2(omega, rho);
  const float2 uu = fma2(ux, ux, mul2(uy, uy));
  const float2 uG = fma2(ux, Gx, mul2(uy, Gy));
  const float2 t = fma2(mul2(splat(-1.5f), orho), uu, mul2(splat(q.kf_m3), uG));

  float2 Cax, Cdg;
  if (WB) {
    const float2 ku = mul2(kf, fma2(ux, grx, mul2(uy, gry)));
    Cax = mul2(splat(1.0f / 9.0f), fma2(half, ku, t));
    Cdg = mul2(splat(1.0f / 36.0f), fma2(splat(2.0f), ku, t));
  } else {
    const float2 s = fma2(omega, rs, t);                 // b_i = w_i rs
    Cax = mul2(splat(1.0f / 9.0f), s);
    Cdg = mul2(splat(1.0f / 36.0f), s);
  }
  const float2 hrho = mul2(half, orho);
  const float2 kGx = mul2(kf, Gx), kGy = mul2(kf, Gy);
  const float2 Mx = fma2(orho, ux, mul2(kf, Fx));
  const float2 My = fma2(orho, uy, mul2(kf, Fy));

  const float2 E1 = fma2(ux, fma2(hrho, ux, kGx), Cax);
  const float2 O1 = mul2(third, Mx);
  const float2 E2 = fma2(uy, fma2(hrho, uy, kGy), Cax);
  const float2 O2 = mul2(third, My);
  const float2 quarter = splat(0.25f), twelfth = splat(1.0f / 12.0f);
  const float2 cu5 = add2(ux, uy);
  const float2 E5 = fma2(mul2(quarter, cu5), fma2(hrho, cu5, add2(kGx, kGy)), Cdg);
  const float2 O5 = mul2(twelfth, add2(Mx, My));
  const float2 cu6 = sub2(uy, ux);
  const float2 E6 = fma2(mul2(quarter, cu6), fma2(hrho, cu6, sub2(kGy, kGx)), Cdg);
  const float2 O6 = mul2(twelfth, sub2(My, Mx));

  const float2 keep = splat(q.keep);
  g[1] = fma2(keep, g[1], add2(E1, O1));
  g[3] = fma2(keep, g[3], sub2(E1, O1));
  g[2] = fma2(keep, g[2], add2(E2, O2));
  g[4] = fma2(keep, g[4], sub2(E2, O2));
  g[5] = fma2(keep, g[5], add2(E5, O5));
  g[7] = fma2(keep, g[7], sub2(E5, O5));
  g[6] = fma2(keep, g[6], add2(E6, O6));
  g[8] = fma2(keep, g[8], sub2(E6, O6));
  if (WB) {
    // node mass balance g_0' = g_0 + (m - a), stochastically rounded.  The
    // moving populations leave as keep g_i + (E +- O), so
    // m - a = (1 - keep) m - 2 (E1 + E2 + E5 + E6) = omega m - 2 sum E, up to
    // their own roundings, which are far below an ulp of g_0.
    float2 h, e;
    const float2 se = add2(add2(E1, E2), add2(E5, E6));
    two_sum2(g[0], fma2(splat(-2.0f), se, mul2(omega, m_in)), h, e);
    g[0] = round_stochastic2(h, e, rnd);
  } else {
    // rest population from the node mass balance, as in the scalar version
    g[0] = sub2(rs, moving_sum2(g));
  }
}

// ---- asynchronous copies into shared memory -------------------------------
//
// The pulled plane rows are copied global -> shared with cp.async (no
// register staging), several rows ahead of use.  Full strips of a lattice
// whose width is a multiple of 4 copy 16-byte chunks (all threads share the
// 9 x (tile_x + 8) / E chunks of a row, E = 16 / sizeof(T)); ragged strips
// and other widths copy element by element.

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async_elem(void* smem, const float* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_elem(void* smem, const double* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// c_iy of direction i (D2Q9 numbering of Sec. II)
__host__ __device__ constexpr int dir_cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

// The three directions of each c_iy class: class 0 (c_iy = 0) {0, 1, 3},
// class 1 (c_iy = +1, pulled from row y-1) {2, 5, 6}, class 2 (c_iy = -1,
// pulled from row y+1) {4, 7, 8}.  All plane rows of one class come from the
// same lattice row, so a copy's row offset depends on its class only.
__host__ __device__ constexpr int class_plane(int cls, int a) {
  return cls == 0 ? (a == 2 ? 3 : a) : (cls == 1 ? (a == 0 ? 2 : a + 4) : (a == 0 ? 4 : a + 6));
}

// Rows kept in the density ring and in the chemical-potential ring.  The
// collision takes rho and grad rho from registers (they are computed with mu
// from the same 3x3 neighbourhood), so the density ring only holds the rows
// the mu pass reads; every ring refill is separated from the last read of
// its slot by a barrier.
constexpr int kRing = 4;
constexpr int kMuRing = 4;

// Staging: each loop iteration advances kRows lattice rows per thread; the
// stage keeps the rows being collided (two behind the density front), the
// kRows rows being reduced to densities, and kAhead groups of kRows rows in
// flight.  min_blocks(tx): resident CTAs the register budget must allow.
template <typename T> struct Staging;
template <> struct Staging<float> {
  static constexpr int kRows = 2;
  static constexpr int kAhead = 2;
  static constexpr int kStages = 2 + kRows + kRows * kAhead;     // 8
  __host__ __device__ static constexpr int min_blocks(int tx) { return 640 / tx > 1 ? 640 / tx : 1; }
  // the batched kernel (case parameters in shared memory) fits the same budget
  __host__ __device__ static constexpr int min_blocks_batch(int tx) { return min_blocks(tx); }
};
template <> struct Staging<double> {
  static constexpr int kRows = 1;
  static constexpr int kAhead = 1;
  static constexpr int kStages = 2 + kRows + kRows * kAhead;     // 4
  __host__ __device__ static constexpr int min_blocks(int tx) { return 65536 / (tx * 128); }
  __host__ __device__ static constexpr int min_blocks_batch(int tx) { return 65536 / (tx * 128); }
};

constexpr int kPad = 4;   // staged columns on each side of a strip (x0-4 .. x0+TX+3)

// Storage offset of column x in the ghost layout of the batched kernel
// (column x at x + ghost_off, its four ghost columns on each side at
// ghost_off - 4 .. ghost_off - 1 and nx + ghost_off .. nx + ghost_off + 3):
// 4, so that a strip's columns and both its halos span the fewest 64-byte
// pieces of a row (9 for 128 float columns).  An offset of 32 floats, which
// makes every warp's 32 stores fill whole 128-byte lines, moved 18 % more
// DRAM reads (the halos then straddle one more piece on each side) and did
// not change the writes.
template <typename T>
__host__ __device__ constexpr int ghost_off() {
  return 4;
}

__host__ __device__ constexpr size_t strip_smem_bytes(int tile, int stages, size_t elem) {
  // 128 bytes of alignment slack + the buffers
  return 128 + ((size_t)stages * 9 + kRing + kMuRing) * (size_t)(tile + 2 * kPad) * elem;
}

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
__host__ __device__ constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }

// The fused step kernel (MOMENTS = false) and the macroscopic-field /
// statistics kernel (MOMENTS = true) share one body so that both evaluate
// rho, mu, F and u with identical arithmetic.
//
// Shared-memory column slot s holds lattice column x0 - 4 + s (wrapped).
// Stage rows hold raw plane rows: stage[slot][i][s] = P_i(x0 - 4 + s, r - c_iy)
// for logical row r, so the pulled population of column s is
// f_i = stage[slot][i][s - c_ix].
//
// Pipeline over the rows k = y0-2 .. y1+1 of a strip (y0..y1-1 are the rows
// this CTA updates), kRows rows per iteration: reduce rows k.. to densities
// (rho ring), request the rows kRows * kAhead further on, compute mu and
// grad rho of rows k-1.. (mu ring; grad rho stays in registers), collide and
// store rows k-2..  Two rows per iteration in FP32 halve the per-row barrier
// and loop overhead and share the stencil loads of neighbouring rows.
//
// Every ring and stage slot repeats after lcm(stages, rings) rows; the row
// loop is unrolled over that period so that all shared-memory offsets are
// compile-time constants, and the strip width TX is a template parameter for
// the same reason.
// blockDim.x = TX; grid = (ceil(nx / TX), ceil(ny / rows)).
// Dynamic shared memory: strip_smem_bytes(TX, kStages, sizeof(T)).
// What one strip pass does with each collided row.
enum StripMode {
  kModeStep = 0,       // store the post-collision populations
  kModeMoments = 1,    // write rho, u, mu fields and per-CTA stats, no store
  kModeStepStats = 2   // store, and accumulate per-CTA stats of f(t)
};

// Per-CTA statistics of the collided nodes (FP64 accumulators).
struct StatsAcc {
  double mass = 0.0, kin = 0.0, u2 = 0.0, mumin = 1e300, mumax = -1e300;
  int bad = 0;
};

// One collided node of row c: store its nine populations (and the ghost
// copies of a boundary column), or write its moment fields, and fold its
// statistics.  Forced inline so that the population array stays in registers.
template <typename T, int MODE, bool GHOST>
__device__ __forceinline__ void emit_node(const KParams& p, const MomentsOut& mo, T* dst, int c,
                                          int xcol, int xm, bool ghost_r, bool ghost_l,
                                          const T (&gv)[9], T rs, T muc, T ux, T uy,
                                          StatsAcc& acc, bool acc_on) {
  constexpr bool MOMENTS = MODE == kModeMoments;
  constexpr bool STATS = MODE != kModeStep;
  if (!MOMENTS && WB_IN(c, p.ny) && WB_IN(xcol, p.pitch)) {
    if (GHOST) {
      // parameters live in shared memory here: one running pointer
      T* o = dst + (unsigned)(c * p.pitch + xcol);
      const long long pl = p.plane;
      const int nx = p.nx;
      const bool gr = ghost_r && WB_IN(xcol + nx, p.pitch);
      const bool gl = ghost_l && WB_IN(xcol - nx, p.pitch);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        *o = gv[i];
        if (gr) o[nx] = gv[i];
        if (gl) o[-nx] = gv[i];
        o += pl;
      }
    } else {
      // kernel parameters: per-plane bases and one 32-bit offset
      const unsigned off = (unsigned)(c * p.pitch + xcol);
#pragma unroll
      for (int i = 0; i < 9; ++i) (dst + i * p.plane)[off] = gv[i];
    }
  }
  if (STATS && acc_on) {
    const double rho = (double)rs + p.rho_ref;
    const double mu = (double)muc;
    const double dux = (double)ux, duy = (double)uy;
    if (MOMENTS && WB_IN(c, p.ny) && WB_IN(xm, p.nx)) {
      const unsigned kk = (unsigned)((c + p.y_offset) * p.nx + xm);
      if (mo.rho) mo.rho[kk] = rho;
      if (mo.ux) mo.ux[kk] = dux;
      if (mo.uy) mo.uy[kk] = duy;
      if (mo.mu) mo.mu[kk] = mu;
    }
    const double u2 = dux * dux + duy * duy;
    acc.mass += rho;
    acc.kin += 0.5 * rho * u2;
    acc.u2 = fmax(acc.u2, u2);
    acc.mumin = fmin(acc.mumin, mu);
    acc.mumax = fmax(acc.mumax, mu);
    if (!isfinite(rho) || !isfinite(mu) || !isfinite(u2)) acc.bad = 1;
  }
}

// GHOST selects the row layout with ghost columns used by the batched
// kernel: column x of a row is stored at x + ghost_off<T>() and the four
// columns on each side hold copies of the wrapped columns (x = -4..-1 ->
// nx-4..nx-1, x = nx..nx+3 -> 0..3), refreshed by every store of a boundary
// column.  A
// strip then reads one contiguous range per plane row, always in 16-byte
// chunks through L2 (cp.async.cg), whatever its width: needed when one
// kernel launch reads data that other CTAs wrote during the same launch (L1
// is not coherent across SMs).  Requires nx >= 8 and
// pitch >= nx + ghost_off + 8.
// Offsets within a plane are 32-bit: pitch * ny < 2^31 (checked by the host).
template <typename T, int SCH, int MODE, int TX, bool GHOST = false>
__device__ __forceinline__ void strip_pass(const T* __restrict__ src, T* __restrict__ dst,
                                           const KParams& p, const MomentsOut& mo, int x0,
                                           int y0, int y1, double* stats_rec,
                                           unsigned char* smem_raw) {
  constexpr bool STATS = MODE != kModeStep;
  constexpr int R = Staging<T>::kRows;     // rows per iteration
  constexpr int PDG = Staging<T>::kAhead;  // row groups requested ahead of use
  constexpr int NST = Staging<T>::kStages;
  constexpr int NPH = lcm_c(lcm_c(NST, kRing), kMuRing) / R;   // iterations per slot period
  static_assert(lcm_c(lcm_c(NST, kRing), kMuRing) % R == 0, "slot period");
  constexpr int SW = TX + 2 * kPad;        // row width of every buffer
  constexpr int E = 16 / sizeof(T);        // elements per 16-byte chunk
  constexpr int NCH = SW / E;              // chunks per plane row (full strip)
  constexpr int CPT = (3 * NCH + TX - 1) / TX;   // chunks per thread and class
  // 128-byte aligned base (16-byte copies need 16)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  T* stage = reinterpret_cast<T*>(base);               // [NST][9][SW]
  T* rho_s = stage + NST * 9 * SW;                     // [kRing][SW]
  T* mu_s = rho_s + kRing * SW;                        // [kMuRing][SW]

  const int tx = threadIdx.x;
  const int w = min(TX, p.nx - x0);        // valid columns of this strip
  const bool own = tx < w;
  __syncthreads();                         // a previous pass may still read smem
  const int sx = tx + kPad;                // slot of the own column
  // Halo work: threads 0-3 take the densities of slots 2, 3 (x0-2, x0-1)
  // and w+4, w+5 (x0+w, x0+w+1); threads mu_lo and mu_hi (warp 1 when there
  // is one) take mu at slots 3 and w+4.  Each halo branch runs in one warp,
  // and the two are in different warps so that no warp carries both.
  const bool halo = tx < 4;
  const int hs = tx < 2 ? 2 + tx : w + 2 + tx;
  constexpr int mu_lo = TX >= 64 ? 32 : 0, mu_hi = mu_lo + 1;
  const bool use_vec = GHOST || ((w == TX) && (p.nx % 4 == 0));
  // 16-byte chunks per plane row this strip needs (its columns plus 4 on
  // each side, rounded up to whole chunks; never past the stage row)
  const int nch_rt = GHOST ? (w + 2 * kPad + E - 1) / E : NCH;

  const T two_beta = T(p.two_beta), dl = T(p.dl), dg = T(p.dg), kappa6 = T(p.kappa / 6.0);
  const CollideConsts<T> cc(p);
  // The second ring holds mu, or lap(rho) with the pressure-form force
  // (chem_pot with beta = 0 and kappa/6 -> -1/6 gives exactly lap(rho)); the
  // gradient carried to the collision is grad(rho), or grad(cs^2 rho - p_0).
  constexpr bool kPress = SCH == kSchPressure;
  const T ring_tb = kPress ? T(0) : two_beta;
  const T ring_k6 = kPress ? T(-1.0 / 6.0) : kappa6;
  const T half_beta = T(0.5 * p.two_beta), rho_ref_t = T(p.rho_ref);
  // cs^2 rho - p_0 from a stored density v (rho = v + rho_ref, up to a
  // constant): p_0 = rho mu_0 - psi_0 = beta a b (2 rho (a + b) - a b),
  // a = rho - rho_l, b = rho - rho_g
  auto press_a = [&](T v) {
    const T a = v + dl, b = v + dg, r = v + rho_ref_t;
    return T(1.0 / 3.0) * v - half_beta * a * b * (T(2) * r * (a + b) - a * b);
  };
  // mu at a node from its stored density and its second-ring value
  auto mu_node = [&](T v, T ringval) {
    if (!kPress) return ringval;
    const T a = v + dl, b = v + dg;
    return two_beta * a * b * (a + b) - cc.kappa * ringval;
  };
  const int kfirst = y0 - 2, klast = y1 + 1;
  // hash key of the time step being taken (stochastic rounding, FP32 WB)
  const uint32_t ht = step_key(p.step + (p.step_base ? *p.step_base : 0LL));

  // 16-byte chunks this thread copies in every row (fixed per thread): in
  // class c, chunk q = tx + m * TX is chunk j of the class's plane a, covering
  // columns x0-4+jE .. x0-4+jE+E-1, which wrap only as a whole (nx % 4 == 0).
  const T* ch_src[3][CPT];
  int ch_dst[3][CPT];
  bool ch_on[3][CPT];
#pragma unroll
  for (int cls = 0; cls < 3; ++cls) {
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const int q = tx + m * TX;
      ch_on[cls][m] = use_vec && q < 3 * nch_rt;
      const int a = ch_on[cls][m] ? q / nch_rt : 0, j = ch_on[cls][m] ? q - a * nch_rt : 0;
      const int i = class_plane(cls, a);
      int col = x0 - kPad + j * E;
      if (GHOST) {
        col += ghost_off<T>();             // storage offset of column x
      } else {
        if (col < 0) col += p.nx;
        else if (col >= p.nx) col -= p.nx;
      }
      ch_src[cls][m] = src + i * p.plane + col;
      ch_dst[cls][m] = i * SW + j * E;
    }
  }

  // Request the next logical row (its plane rows r - c_iy) into stage slot
  // `slot`.  Rows are requested in order kfirst, kfirst+1, ...; the wrapped
  // row index and the offsets of rows r+1, r, r-1 advance incrementally.
  int req_rw = wrap_index(kfirst, p.ny);
  int row_p = ((req_rw == p.ny - 1) ? 0 : req_rw + 1) * p.pitch;
  int row_0 = req_rw * p.pitch;
  int row_m = ((req_rw == 0) ? p.ny - 1 : req_rw - 1) * p.pitch;
  // Rows kfirst .. kfirst + nlast are processed in groups of R (a row past
  // klast only feeds values nobody reads).
  const int ngroups = (klast - kfirst + R) / R;
  const int nlast = R * ngroups - 1;       // last row, relative to kfirst
  auto request_next = [&](int slot) {
    T* st = stage + slot * 9 * SW;
    if (use_vec) {
#pragma unroll
      for (int cls = 0; cls < 3; ++cls) {
        const int roff = cls == 0 ? row_0 : (cls == 1 ? row_m : row_p);
#pragma unroll
        for (int m = 0; m < CPT; ++m)
          if (ch_on[cls][m] && WB_IN(ch_src[cls][m] + roff - src, 9 * p.plane - (E - 1)) &&
              WB_IN(ch_dst[cls][m], 9 * SW - (E - 1)))
            cp_async16(st + ch_dst[cls][m], ch_src[cls][m] + roff);
      }
    } else {
      const int ncols = w + 2 * kPad;
      for (int j = tx; j < ncols; j += TX) {
        const int col = wrap_index(x0 - kPad + j, p.nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int roff = dir_cy(i) == -1 ? row_p : (dir_cy(i) == 0 ? row_0 : row_m);
          if (WB_IN(i * p.plane + roff + col, 9 * p.plane) && WB_IN(j, SW))
            cp_async_elem(st + i * SW + j, src + i * p.plane + roff + col);
        }
      }
    }
    req_rw = (req_rw + 1 == p.ny) ? 0 : req_rw + 1;
    row_m = row_0;
    row_0 = row_p;
    row_p = ((req_rw + 1 == p.ny) ? 0 : req_rw + 1) * p.pitch;
  };
  // density of the staged row at slot s: sum_i f_i, f_i = stage[i][s - c_ix]
  auto staged_rho = [&](const T* st, int s) {
    return ((st[0 * SW + s] + st[1 * SW + s - 1]) + (st[2 * SW + s] + st[3 * SW + s + 1])) +
           ((st[4 * SW + s] + st[5 * SW + s - 1]) + (st[6 * SW + s + 1] + st[7 * SW + s + 1])) +
           st[8 * SW + s - 1];
  };



  // store position of column x0 + tx within a plane; ghost copies a boundary
  // column also writes: x < 4 -> +nx (right ghost), x >= nx - 4 -> -nx (left)
  const int xcol = x0 + tx + (GHOST ? ghost_off<T>() : 0);
  const int xg = x0 + tx;
  const bool ghost_r = GHOST && own && xg < kPad;
  const bool ghost_l = GHOST && own && xg >= p.nx - kPad;

  {
    int sq = 0;                            // stage slot of the next requested row
    for (int gq = 0; gq < PDG; ++gq) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (gq * R + j <= nlast) request_next(sq);
        ++sq;
      }
      cp_async_commit();                   // one group per R rows, possibly empty
    }
  }
  cp_async_wait<PDG - 1>();                // first group landed (this thread)
  __syncthreads();                         // ... and everyone else's

  StatsAcc acc;
  const int xm = x0 + tx;                  // column of the moment fields
  // statistics are gathered only into a record (a uniform, runtime choice in
  // the step-and-statistics mode, so that one instantiation serves both)
  const bool acc_on = MODE == kModeMoments || stats_rec != nullptr;

  // FP32: the two rows of an iteration run as float2 pairs
  constexpr bool kPacked = sizeof(T) == 4 && R == 2;
  // rho and grad rho of the last mu row(s) of the previous iteration
  T prs = T(0), pgx = T(0), pgy = T(0);
  // x-neighbour density sums of the own column in the rows below the
  // density front (scalar path: rows n0-1 and n0-2)
  T psum_c = T(0), psum_b = T(0);
  T pdif_c = T(0), pdif_b = T(0);          // ... and x-differences (grad rho)
  float2 prs2 = make_float2(0.f, 0.f), pgx2 = prs2, pgy2 = prs2;
  const float2 tb2 = make_float2((float)ring_tb, (float)ring_tb);
  const float2 dl2 = make_float2((float)dl, (float)dl), dg2 = make_float2((float)dg, (float)dg);
  const float2 k62 = make_float2((float)ring_k6, (float)ring_k6);
  auto press_a2 = [&](float2 v) { return make_float2((float)press_a(T(v.x)), (float)press_a(T(v.y))); };
  // pair (lo[s], hi[s]) of two buffer rows
  auto V = [](const T* lo, const T* hi, int s) { return make_float2((float)lo[s], (float)hi[s]); };
  bool live = true;
  for (int n = 0; live; n += NPH * R) {
#pragma unroll
    for (int ph = 0; ph < NPH; ++ph) {
      const int n0 = n + ph * R;           // density front, relative to kfirst
      if (live && n0 > nlast) live = false;
      if (live) {
        // slot of the row at relative offset d from this iteration's front
        // (ph * R + d, taken modulo the ring; compile-time after unrolling)
#define WB_SLOT(d, ring) ((ph * R + (d) + 4 * (ring)) % (ring))
        if constexpr (kPacked) {
          const T* s0 = stage + WB_SLOT(0, NST) * 9 * SW;
          const T* s1 = stage + WB_SLOT(1, NST) * 9 * SW;
          T* r0 = rho_s + WB_SLOT(0, kRing) * SW;
          T* r1 = rho_s + WB_SLOT(1, kRing) * SW;
          // rho = g_0 + (moving sum, mirror-symmetric grouping): the same two
          // operations collide_x2 repeats for the exact mass balance
          auto rho2 = [&](int s) {
            const float2 m = add2(add2(add2(V(s0, s1, 1 * SW + s - 1), V(s0, s1, 3 * SW + s + 1)),
                                       add2(V(s0, s1, 2 * SW + s), V(s0, s1, 4 * SW + s))),
                                  add2(add2(V(s0, s1, 5 * SW + s - 1), V(s0, s1, 7 * SW + s + 1)),
                                       add2(V(s0, s1, 6 * SW + s + 1), V(s0, s1, 8 * SW + s - 1))));
            return add2(V(s0, s1, 0 * SW + s), m);
          };
          if (own) {
            const float2 v = rho2(sx);
            if (halo) {
              const float2 h = rho2(hs);
              if (WB_IN(hs, SW)) {
                r0[hs] = h.x;
                r1[hs] = h.y;
              }
            }
            r0[sx] = v.x;
            r1[sx] = v.y;
          } else if (halo) {
            const float2 h = rho2(hs);
            if (WB_IN(hs, SW)) {
              r0[hs] = h.x;
              r1[hs] = h.y;
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const T* st = stage + WB_SLOT(j, NST) * 9 * SW;
            T* row = rho_s + WB_SLOT(j, kRing) * SW;
            if (own) row[sx] = staged_rho(st, sx);
            if (halo && WB_IN(hs, SW)) row[hs] = staged_rho(st, hs);
          }
        }
        // barrier B: every read of the stage slots about to be refilled (rows
        // collided an iteration ago) and of the mu ring rows about to be
        // rewritten is done
        __syncthreads();
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (n0 + R * PDG + j <= nlast) request_next(WB_SLOT(R * PDG + j, NST));
        cp_async_commit();
        cp_async_wait<PDG - 1>();          // next group landed (visible after barrier C)

        // mu (ring) and rho, grad rho (registers) of rows n0-1+j
        T frs[R], fgx[R], fgy[R];
        float2 frs2 = make_float2(0.f, 0.f), fgx2 = frs2, fgy2 = frs2;
        if constexpr (kPacked) {
          // lane x: row n0-1, lane y: row n0 (rows below n0-1 feed nothing)
          if (kfirst + n0 >= y0 - 1) {
            const T* rb = rho_s + WB_SLOT(-2, kRing) * SW;   // row n0-2
            const T* rc = rho_s + WB_SLOT(-1, kRing) * SW;   // row n0-1
            const T* ra = rho_s + WB_SLOT(0, kRing) * SW;    // row n0
            const T* rt = rho_s + WB_SLOT(1, kRing) * SW;    // row n0+1
            T* m0 = mu_s + WB_SLOT(-1, kMuRing) * SW;
            T* m1 = mu_s + WB_SLOT(0, kMuRing) * SW;
            auto at2 = [&](int s) {
              return chem_pot_x2(V(rc, ra, s), V(rc, ra, s + 1), V(rc, ra, s - 1), V(ra, rt, s),
                                 V(rb, rc, s), V(ra, rt, s + 1), V(ra, rt, s - 1),
                                 V(rb, rc, s + 1), V(rb, rc, s - 1), tb2, dl2, dg2, k62);
            };
            if (own) {
              // all loads before the ring stores, so that they are shared
              const float2 mu = at2(sx);
              frs2 = V(rc, ra, sx);
              if (kPress)
                iso_grad_x2(press_a2(V(rc, ra, sx + 1)), press_a2(V(rc, ra, sx - 1)),
                            press_a2(V(ra, rt, sx)), press_a2(V(rb, rc, sx)),
                            press_a2(V(ra, rt, sx + 1)), press_a2(V(ra, rt, sx - 1)),
                            press_a2(V(rb, rc, sx + 1)), press_a2(V(rb, rc, sx - 1)), fgx2, fgy2);
              else
                iso_grad_x2(V(rc, ra, sx + 1), V(rc, ra, sx - 1), V(ra, rt, sx), V(rb, rc, sx),
                            V(ra, rt, sx + 1), V(ra, rt, sx - 1), V(rb, rc, sx + 1),
                            V(rb, rc, sx - 1), fgx2, fgy2);
              m0[sx] = mu.x;
              m1[sx] = mu.y;
            }
            if (tx == mu_lo || tx == mu_hi) {   // halo mu at slots 3 and w+4
              const int s = tx == mu_lo ? 3 : w + 4;
              const float2 mu = at2(s);
              if (WB_IN(s, SW)) {
                m0[s] = mu.x;
                m1[s] = mu.y;
              }
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < R; ++j) {
            frs[j] = fgx[j] = fgy[j] = T(0);
            const T* rn = rho_s + WB_SLOT(j, kRing) * SW;         // row above (y+1)
            // x-neighbour sum and difference of the density row just
            // reduced, carried to the mu rows of the next two iterations
            const T psum_n = own ? rn[sx + 1] + rn[sx - 1] : T(0);
            const T pdif_n = (own && !kPress) ? rn[sx + 1] - rn[sx - 1] : T(0);
            if (kfirst + n0 - 1 + j >= y0 - 1) {
              const T* rc = rho_s + WB_SLOT(j - 1, kRing) * SW;
              const T* rsb = rho_s + WB_SLOT(j - 2, kRing) * SW;  // row below (y-1)
              T* mrow = mu_s + WB_SLOT(j - 1, kMuRing) * SW;
              auto at = [&](int s) {
                return chem_pot<T>(rc[s], rc[s + 1], rc[s - 1], rn[s], rsb[s], rn[s + 1],
                                   rn[s - 1], rsb[s + 1], rsb[s - 1], ring_tb, dl, dg, ring_k6);
              };
              if (own) {
                mrow[sx] = chem_pot_rows<T>(rc[sx], psum_c, rn[sx], rsb[sx], psum_n, psum_b,
                                            ring_tb, dl, dg, ring_k6);
                frs[j] = rc[sx];
                // 12 grad(rho) (or 12 grad(cs^2 rho - p_0)): see iso_grad12
                // and iso_grad12_rows
                if (kPress)
                  iso_grad12<T>(press_a(rc[sx + 1]), press_a(rc[sx - 1]), press_a(rn[sx]),
                                press_a(rsb[sx]), press_a(rn[sx + 1]), press_a(rn[sx - 1]),
                                press_a(rsb[sx + 1]), press_a(rsb[sx - 1]), fgx[j], fgy[j]);
                else
                  iso_grad12_rows<T>(pdif_c, pdif_n, pdif_b, rn[sx], rsb[sx], psum_n, psum_b,
                                     fgx[j], fgy[j]);
              }
              if (tx == mu_lo) mrow[3] = at(3);
              if (tx == mu_hi && WB_IN(w + 4, SW)) mrow[w + 4] = at(w + 4);
            }
            psum_b = psum_c;
            psum_c = psum_n;
            pdif_b = pdif_c;
            pdif_c = pdif_n;
          }
        }
        __syncthreads();                   // barrier C

        if constexpr (kPacked) {
          const int c0 = kfirst + n0 - 2;    // rows c0 (lane x) and c0+1 (lane y)
          const bool v0 = c0 >= y0 && c0 < y1, v1 = c0 + 1 >= y0 && c0 + 1 < y1;
          if (own && (v0 || v1)) {
            const T* mA = mu_s + WB_SLOT(-3, kMuRing) * SW;    // row c0-1
            const T* mB = mu_s + WB_SLOT(-2, kMuRing) * SW;    // row c0
            const T* mC = mu_s + WB_SLOT(-1, kMuRing) * SW;    // row c0+1
            const T* mD = mu_s + WB_SLOT(0, kMuRing) * SW;     // row c0+2
            float2 gmx, gmy;
            iso_grad_x2(V(mB, mC, sx + 1), V(mB, mC, sx - 1), V(mC, mD, sx), V(mA, mB, sx),
                        V(mC, mD, sx + 1), V(mC, mD, sx - 1), V(mA, mB, sx + 1),
                        V(mA, mB, sx - 1), gmx, gmy);
            // rho, grad rho of row c0 come from the previous iteration's lane y
            const float2 rs = make_float2(prs2.y, frs2.x);
            const float2 grx = make_float2(pgx2.y, fgx2.x), gry = make_float2(pgy2.y, fgy2.x);
            const T* s0 = stage + WB_SLOT(-2, NST) * 9 * SW;
            const T* s1 = stage + WB_SLOT(-1, NST) * 9 * SW;
            // f_i(x) = P_i(x - c_i): column offset -c_ix within the staged rows
            float2 g[9] = {V(s0, s1, 0 * SW + sx),     V(s0, s1, 1 * SW + sx - 1),
                           V(s0, s1, 2 * SW + sx),     V(s0, s1, 3 * SW + sx + 1),
                           V(s0, s1, 4 * SW + sx),     V(s0, s1, 5 * SW + sx - 1),
                           V(s0, s1, 6 * SW + sx + 1), V(s0, s1, 7 * SW + sx + 1),
                           V(s0, s1, 8 * SW + sx - 1)};
            float2 ux, uy;
            // draws of rows c0 and c0 + 1 (one hash when the global row of
            // c0 is even, the usual case; its parity is fixed within a CTA)
            const int cg = c0 + p.y_offset;
            const uint32_t kx = (uint32_t)cg * (uint32_t)p.nx + (uint32_t)xm;
            float2 rnd;
            if ((cg & 1) == 0) {
              rnd = pair_uniforms(kx, ht);
            } else {
              rnd = make_float2(pair_uniforms(kx - (uint32_t)p.nx, ht).y,
                                pair_uniforms(kx + (uint32_t)p.nx, ht).x);
            }
            collide_x2<SCH>(g, rs, gmx, gmy, grx, gry, cc, ux, uy, rnd);
            if (v0) {
              const T gl[9] = {g[0].x, g[1].x, g[2].x, g[3].x, g[4].x,
                               g[5].x, g[6].x, g[7].x, g[8].x};
              emit_node<T, MODE, GHOST>(p, mo, dst, c0, xcol, xm, ghost_r, ghost_l, gl, rs.x,
                                        STATS ? mu_node(rs.x, mB[sx]) : T(0), ux.x, uy.x, acc, acc_on);
            }
            if (v1) {
              const T gh[9] = {g[0].y, g[1].y, g[2].y, g[3].y, g[4].y,
                               g[5].y, g[6].y, g[7].y, g[8].y};
              emit_node<T, MODE, GHOST>(p, mo, dst, c0 + 1, xcol, xm, ghost_r, ghost_l, gh,
                                        rs.y, STATS ? mu_node(rs.y, mC[sx]) : T(0), ux.y, uy.y, acc, acc_on);
            }
          }
          prs2 = frs2;
          pgx2 = fgx2;
          pgy2 = fgy2;
        } else {
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int c = kfirst + n0 - 2 + j;   // row to collide
            if (c >= y0 && c < y1 && own) {
              const T* m_dn = mu_s + WB_SLOT(j - 3, kMuRing) * SW;
              const T* m_c = mu_s + WB_SLOT(j - 2, kMuRing) * SW;
              const T* m_up = mu_s + WB_SLOT(j - 1, kMuRing) * SW;
              // "up" is row c+1 (+y), "dn" row c-1; slot sx+1 is +x
              T gmx, gmy;                        // 12 grad(mu)
              iso_grad12<T>(m_c[sx + 1], m_c[sx - 1], m_up[sx], m_dn[sx], m_up[sx + 1],
                            m_up[sx - 1], m_dn[sx + 1], m_dn[sx - 1], gmx, gmy);
              const T rs = j == 0 ? prs : frs[j - 1];
              const T grx = j == 0 ? pgx : fgx[j - 1];
              const T gry = j == 0 ? pgy : fgy[j - 1];
              const T* st = stage + WB_SLOT(j - 2, NST) * 9 * SW;
              // f_i(x) = P_i(x - c_i): column offset -c_ix within the staged rows
              T g[9] = {st[0 * SW + sx],     st[1 * SW + sx - 1], st[2 * SW + sx],
                        st[3 * SW + sx + 1], st[4 * SW + sx],     st[5 * SW + sx - 1],
                        st[6 * SW + sx + 1], st[7 * SW + sx + 1], st[8 * SW + sx - 1]};
              T ux, uy;
              collide<T, SCH, 12>(g, rs, gmx, gmy, grx, gry, cc, ux, uy);
              emit_node<T, MODE, GHOST>(p, mo, dst, c, xcol, xm, ghost_r, ghost_l, g, rs,
                                        STATS ? mu_node(rs, m_c[sx]) : T(0), ux, uy, acc, acc_on);
            }
          }
          prs = frs[R - 1];
          pgx = fgx[R - 1];
          pgy = fgy[R - 1];
        }
#undef WB_SLOT
      }
    }
  }
  cp_async_wait<0>();

  if (STATS && stats_rec) {
    // deterministic block reduction: warp shuffle, then thread 0 over warps
    __shared__ double red[kMaxTile / 32][kStatRec];
    double v[kStatRec] = {acc.mass, acc.kin, acc.u2, acc.mumin, acc.mumax, (double)acc.bad};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double o0 = __shfl_down_sync(0xffffffffu, v[0], off);
      double o1 = __shfl_down_sync(0xffffffffu, v[1], off);
      double o2 = __shfl_down_sync(0xffffffffu, v[2], off);
      double o3 = __shfl_down_sync(0xffffffffu, v[3], off);
      double o4 = __shfl_down_sync(0xffffffffu, v[4], off);
      double o5 = __shfl_down_sync(0xffffffffu, v[5], off);
      v[0] += o0;
      v[1] += o1;
      v[2] = fmax(v[2], o2);
      v[3] = fmin(v[3], o3);
      v[4] = fmax(v[4], o4);
      v[5] = fmax(v[5], o5);
    }
    const int warp = tx >> 5, lane = tx & 31, nw = TX >> 5;
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) red[warp][q] = v[q];
    __syncthreads();
    if (tx == 0) {
      double r[kStatRec];
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) r[q] = red[0][q];
      for (int q = 1; q < nw; ++q) {
        r[0] += red[q][0];
        r[1] += red[q][1];
        r[2] = fmax(r[2], red[q][2]);
        r[3] = fmin(r[3], red[q][3]);
        r[4] = fmax(r[4], red[q][4]);
        r[5] = fmax(r[5], red[q][5]);
      }
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) stats_rec[q] = r[q];
    }
  }
}

// One CTA per strip segment: blockIdx.x picks the strip, blockIdx.y the run
// of p.rows rows (from p.row_lo).  MODE is a StripMode: the moments mode, and the step with
// statistics (a step that also reduces the stats of the state it starts
// from), write the per-CTA stats record.
template <typename T, int SCH, int MODE, int TX>
__global__ void __launch_bounds__(TX, Staging<T>::min_blocks(TX))
    lbm_strip_kernel(const T* __restrict__ src, T* __restrict__ dst,
                     const KParams p, const MomentsOut mo) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int x0 = blockIdx.x * TX;
  const int y0 = p.row_lo + blockIdx.y * p.rows;
  const int y1 = min(y0 + p.rows, p.row_hi);
  double* rec = (MODE != kModeStep && mo.partials)
                    ? mo.partials + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kStatRec
                    : nullptr;
  strip_pass<T, SCH, MODE, TX>(src, dst, p, mo, x0, y0, y1, rec, smem_raw);
}

// Final reduction of the per-CTA records, one block, fixed order.
// out: mass, kinetic, umax, mu_min, mu_max, nonfinite.  (static: every
// translation unit that includes this header gets its own copy.)
static __global__ void __launch_bounds__(256)
    stats_finalize_kernel(const double* __restrict__ partials, int n,
                          double* __restrict__ out) {
  __shared__ double red[256][kStatRec];
  const int t = threadIdx.x;
  double v[kStatRec] = {0.0, 0.0, 0.0, 1e300, -1e300, 0.0};
  for (int k = t; k < n; k += blockDim.x) {
    const double* r = partials + (size_t)k * kStatRec;
    v[0] += r[0];
    v[1] += r[1];
    v[2] = fmax(v[2], r[2]);
    v[3] = fmin(v[3], r[3]);
    v[4] = fmax(v[4], r[4]);
    v[5] = fmax(v[5], r[5]);
  }
#pragma unroll
  for (int k = 0; k < kStatRec; ++k) red[t][k] = v[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) {
      red[t][0] += red[t + s][0];
      red[t][1] += red[t + s][1];
      red[t][2] = fmax(red[t][2], red[t + s][2]);
      red[t][3] = fmin(red[t][3], red[t + s][3]);
      red[t][4] = fmax(red[t][4], red[t + s][4]);
      red[t][5] = fmax(red[t][5], red[t + s][5]);
    }
    __syncthreads();
  }
  if (t == 0) {
    out[0] = red[0][0];
    out[1] = red[0][1];
    out[2] = sqrt(red[0][2]);
    out[3] = red[0][3];
    out[4] = red[0][4];
    out[5] = red[0][5];
  }
}

// Per-direction constants for the layout kernels.
static __constant__ int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static __constant__ int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Initial state f_i = f_i^eq(rho, u = 0), stored for pull streaming:
// P_i(y) = f_i(y + c_i) - s_i.  rest0 / rest_i: the rest equilibrium as
// a function of rho (std: w_i rho; WB: rho - (1-w0) rho0 and w_i rho0);
// shift_i: s_i (0 in FP64).
struct LayoutParams {
  int nx, ny, pitch;
  long long plane;
  int wb;                 // 1: well-balanced rest state
  double rho0;
  double shift[9];
};

template <typename T>
__global__ void init_rest_kernel(const double* __restrict__ rho, T* __restrict__ dst,
                                 const LayoutParams lp) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= lp.nx) return;
  const double w[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int sxw = wrap_index(x + kCx[i], lp.nx);
    const int syw = wrap_index(y + kCy[i], lp.ny);
    const double r = rho[(size_t)syw * lp.nx + sxw];
    double fe;
    if (lp.wb)
      fe = (i == 0) ? r - (1.0 - w[0]) * lp.rho0 : w[i] * lp.rho0;
    else
      fe = w[i] * r;
    dst[i * lp.plane + (long long)y * lp.pitch + x] = (T)(fe - lp.shift[i]);
  }
}

// Populations out: f[i][y][x] = P_i(x - c_i) + s_i as float64.
template <typename T>
__global__ void get_pops_kernel(const T* __restrict__ src, double* __restrict__ f,
                                const LayoutParams lp, int first_dir, int ndir) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= lp.nx) return;
  for (int d = 0; d < ndir; ++d) {
    const int i = first_dir + d;
    const int sxw = wrap_index(x - kCx[i], lp.nx);
    const int syw = wrap_index(y - kCy[i], lp.ny);
    const double v = (double)src[i * lp.plane + (long long)syw * lp.pitch + sxw];
    f[(size_t)d * lp.nx * lp.ny + (size_t)y * lp.nx + x] = v + lp.shift[i];
  }
}

// Populations in: P_i(y) = f_i(y + c_i) - s_i.
template <typename T>
__global__ void set_pops_kernel(const double* __restrict__ f, T* __restrict__ dst,
                                const LayoutParams lp, int first_dir, int ndir) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= lp.nx) return;
  for (int d = 0; d < ndir; ++d) {
    const int i = first_dir + d;
    const int sxw = wrap_index(x + kCx[i], lp.nx);
    const int syw = wrap_index(y + kCy[i], lp.ny);
    const double v = f[(size_t)d * lp.nx * lp.ny + (size_t)syw * lp.nx + sxw];
    dst[i * lp.plane + (long long)y * lp.pitch + x] = (T)(v - lp.shift[i]);
  }
}

}  // namespace wblbe
