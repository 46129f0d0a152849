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
// upward.  For every row it pulls the nine populations of its columns (one
// thread per column, coalesced along x) plus two halo columns on each side
// into shared memory with asynchronous copies issued several rows ahead,
// reduces them to the density (Eq. rhoU) and keeps the densities of the
// last rows in a shared-memory ring.  The chemical potential
// mu = mu_0(rho) - kappa lap(rho) of the row below is computed into a second
// ring, and the row two below the load front is collided: gradients of mu
// and rho (isotropic central stencil), the interaction force (Eq. mF or the
// potential form of Sec. II), the velocity (Eq. rhoU), the equilibrium and
// forcing terms (Eq. mFeq/mFi or Eq. feq/Fi) and the BGK update are all
// evaluated in registers, and the nine results are stored to the other
// buffer.  Each population is read from DRAM once per step (the halo rows and
// columns of neighbouring strips come from L2), and written once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wblbe {

constexpr int kRing = 8;          // rows kept in each shared-memory ring
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
  double wb_b0c;                  // WB: (1 - w0) rho0 in FP64 storage, else 0
  double wb_bax, wb_bdg;          // WB: w_axis rho0, w_diag rho0 (FP64), else 0
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

__device__ __forceinline__ int wrap_index(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// mu = mu_0(rho) - kappa lap(rho) at one node from the 3x3 neighbourhood of
// stored densities rs (rho = rs + rho_ref):
//   mu_0 = 2 beta (rho - rho_l)(rho - rho_g)(2 rho - rho_l - rho_g)
//   lap  = [4 (E + W + N + S) + (NE + NW + SE + SW) - 20 C] / 6
template <typename T>
__device__ __forceinline__ T chem_pot(T c, T e, T w, T n, T s, T ne, T nw, T se,
                                      T sw, T two_beta, T dl, T dg, T kappa) {
  T a = c + dl, b = c + dg;
  T mu0 = two_beta * a * b * (a + b);
  T lap = (T(4) * ((e + w) + (n + s)) + ((ne + nw) + (se + sw)) - T(20) * c) *
          T(1.0 / 6.0);
  return mu0 - kappa * lap;
}

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
// part O of  omega feq_i + kforce F_i.
template <typename T, bool WB>
__device__ __forceinline__ void collide(T (&g)[9], T rs, T gmx, T gmy, T grx,
                                        T gry, const KParams& p, T& ux_out,
                                        T& uy_out) {
  const T omega = T(p.omega), kf = T(p.kforce);
  const T rho = rs + T(p.rho_ref);
  T Fx, Fy;
  if (WB) {
    Fx = -rho * gmx;                                     // Eq. mF
    Fy = -rho * gmy;
  } else {
    Fx = T(1.0 / 3.0) * grx - rho * gmx;                 // potential form
    Fy = T(1.0 / 3.0) * gry - rho * gmy;
  }
  const T jx = ((g[1] - g[3]) + (g[5] - g[7])) + (g[8] - g[6]);
  const T jy = ((g[2] - g[4]) + (g[5] - g[7])) + (g[6] - g[8]);
  const T inv_rho = T(1) / rho;
  const T ux = (jx + T(0.5) * Fx) * inv_rho;            // Eq. rhoU
  const T uy = (jy + T(0.5) * Fy) * inv_rho;
  ux_out = ux;
  uy_out = uy;

  T Gx = Fx, Gy = Fy, ugr = T(0);
  if (WB) {
    Gx = Fx + T(1.0 / 3.0) * grx;
    Gy = Fy + T(1.0 / 3.0) * gry;
    ugr = ux * grx + uy * gry;
  }
  const T uu = ux * ux + uy * uy;
  const T A = T(-1.5) * uu;                  // -3/2 u.u
  const T B = T(-3) * (ux * Gx + uy * Gy);   // -3 u.G
  const T orho = omega * rho;

  // base terms
  T b0, bax, bdg;
  if (WB) {
    b0 = rs - T(p.wb_b0c);
    bax = T(p.wb_bax);
    bdg = T(p.wb_bdg);
  } else {
    b0 = T(4.0 / 9.0) * rs;
    bax = T(1.0 / 9.0) * rs;
    bdg = T(1.0 / 36.0) * rs;
  }
  const T keep = T(1) - omega;

  // rest direction: w0 = 4/9, h0 = -1 (WB)
  const T E0 = omega * b0 + T(4.0 / 9.0) * (orho * A + kf * (B - ugr));
  // axis directions: w = 1/9, h = 1/2 (WB)
  const T Cax = omega * bax + T(1.0 / 9.0) * (orho * A + kf * (B + T(0.5) * ugr));
  // diagonal directions: w = 1/36, h = 2 (WB)
  const T Cdg = omega * bdg + T(1.0 / 36.0) * (orho * A + kf * (B + T(2) * ugr));
  const T hrho = T(0.5) * orho;              // (omega rho / 9) * 9/2
  const T Mx = orho * ux + kf * Fx;          // odd parts: omega rho c.u + kf c.F
  const T My = orho * uy + kf * Fy;

  // pair (1,3): c = (1,0)
  const T E1 = Cax + ux * (hrho * ux + kf * Gx);
  const T O1 = T(1.0 / 3.0) * Mx;
  // pair (2,4): c = (0,1)
  const T E2 = Cax + uy * (hrho * uy + kf * Gy);
  const T O2 = T(1.0 / 3.0) * My;
  // pair (5,7): c = (1,1)
  const T cu5 = ux + uy, cG5 = Gx + Gy;
  const T E5 = Cdg + T(0.25) * cu5 * (hrho * cu5 + kf * cG5);
  const T O5 = T(1.0 / 12.0) * (Mx + My);
  // pair (6,8): c = (-1,1)
  const T cu6 = uy - ux, cG6 = Gy - Gx;
  const T E6 = Cdg + T(0.25) * cu6 * (hrho * cu6 + kf * cG6);
  const T O6 = T(1.0 / 12.0) * (My - Mx);

  g[0] = keep * g[0] + E0;
  g[1] = keep * g[1] + (E1 + O1);
  g[3] = keep * g[3] + (E1 - O1);
  g[2] = keep * g[2] + (E2 + O2);
  g[4] = keep * g[4] + (E2 - O2);
  g[5] = keep * g[5] + (E5 + O5);
  g[7] = keep * g[7] + (E5 - O5);
  g[6] = keep * g[6] + (E6 + O6);
  g[8] = keep * g[8] + (E6 - O6);
}

// Asynchronous global -> shared copies (cp.async, sm_80 and later).  The
// pulled populations of a row are copied into shared memory several rows
// ahead of their use, so the data in flight occupies no registers.
__device__ __forceinline__ void cp_async_elem(void* smem, const float* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(void* smem, const double* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rows of populations staged in shared memory: the pipeline keeps the row
// being collided, the two rows above it, and kStages - 3 rows in flight.
template <typename T> struct Staging;
template <> struct Staging<float> { static constexpr int kStages = 8; };
template <> struct Staging<double> { static constexpr int kStages = 4; };

__host__ __device__ constexpr size_t strip_smem_bytes(int tile, int stages, size_t elem) {
  return ((size_t)stages * 9 + 2 * kRing) * (size_t)(tile + 2 * kHalo) * elem;
}

// The fused step kernel (MOMENTS = false) and the macroscopic-field /
// statistics kernel (MOMENTS = true) share one body so that both evaluate
// rho, mu, F and u with identical arithmetic.
//
// Pipeline over the rows k = y0-2 .. y1+1 of a strip (y0..y1-1 are the rows
// this CTA updates): row k + PD is requested (cp.async, already pulled:
// stage[i][slot] = P_i(x - c_i)), row k's density goes to the rho ring,
// mu of row k-1 to the mu ring, and row k-2 is collided and stored.  Every
// staged element is written and read by the same thread, so only the two
// rings need barriers.
//
// blockDim.x = tile_x; grid = (ceil(nx / tile_x), ceil(ny / rows)).
// Dynamic shared memory: strip_smem_bytes(tile_x, kStages, sizeof(T)).
template <typename T, bool WB, bool MOMENTS>
__global__ void __launch_bounds__(kMaxTile)
    lbm_strip_kernel(const T* __restrict__ src, T* __restrict__ dst,
                     const KParams p, const MomentsOut mo) {
  constexpr int kStages = Staging<T>::kStages;
  constexpr int PD = kStages - 3;          // rows requested ahead of use
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = blockDim.x;
  const int SW = TX + 2 * kHalo;           // row width of every buffer
  T* stage = reinterpret_cast<T*>(smem_raw);          // [kStages][9][SW]
  T* rho_s = stage + kStages * 9 * SW;                 // [kRing][SW]
  T* mu_s = rho_s + kRing * SW;                        // [kRing][SW]

  const int tx = threadIdx.x;
  const int x0 = blockIdx.x * TX;
  const int w = min(TX, p.nx - x0);        // valid columns of this strip
  const int y0 = blockIdx.y * p.rows;
  const int y1 = min(y0 + p.rows, p.ny);
  const bool own = tx < w;

  // Columns this thread pulls: its own column (tx < w) and, for tx < 4, one
  // halo column (slots 0, 1 and w+2, w+3).
  const int xc = own ? x0 + tx : x0;
  const int xl = (xc == 0) ? p.nx - 1 : xc - 1;
  const int xr = (xc == p.nx - 1) ? 0 : xc + 1;
  const bool halo = tx < 2 * kHalo;
  int hs = 0, hc = 0, hl = 0, hr = 0;
  if (halo) {
    hs = tx < kHalo ? tx : w + tx;
    const int gx = x0 - kHalo + hs;        // may lie outside [0, nx)
    hc = wrap_index(gx, p.nx);
    hl = wrap_index(gx - 1, p.nx);
    hr = wrap_index(gx + 1, p.nx);
  }
  const int sx = tx + kHalo;

  const T two_beta = T(p.two_beta), dl = T(p.dl), dg = T(p.dg), kappa = T(p.kappa);

  // Request the pulled populations of lattice row r (logical, may lie
  // outside [0, ny)) into its stage slot:  f_i(x, r) = P_i(x - c_i, r - c_iy).
  auto request = [&](int r) {
    const int rw = wrap_index(r, p.ny);
    const int rm = ((rw == 0) ? p.ny - 1 : rw - 1) * p.pitch;   // row r - 1
    const int r0 = rw * p.pitch;
    const int rp = ((rw == p.ny - 1) ? 0 : rw + 1) * p.pitch;   // row r + 1
    T* st = stage + (r & (kStages - 1)) * 9 * SW;
    auto pull = [&](int s, int cl, int cc, int cr) {
      cp_async_elem(st + 0 * SW + s, src + 0 * p.plane + r0 + cc);
      cp_async_elem(st + 1 * SW + s, src + 1 * p.plane + r0 + cl);   // c1 = ( 1, 0)
      cp_async_elem(st + 2 * SW + s, src + 2 * p.plane + rm + cc);   // c2 = ( 0, 1)
      cp_async_elem(st + 3 * SW + s, src + 3 * p.plane + r0 + cr);   // c3 = (-1, 0)
      cp_async_elem(st + 4 * SW + s, src + 4 * p.plane + rp + cc);   // c4 = ( 0,-1)
      cp_async_elem(st + 5 * SW + s, src + 5 * p.plane + rm + cl);   // c5 = ( 1, 1)
      cp_async_elem(st + 6 * SW + s, src + 6 * p.plane + rm + cr);   // c6 = (-1, 1)
      cp_async_elem(st + 7 * SW + s, src + 7 * p.plane + rp + cr);   // c7 = (-1,-1)
      cp_async_elem(st + 8 * SW + s, src + 8 * p.plane + rp + cl);   // c8 = ( 1,-1)
    };
    if (own) pull(sx, xl, xc, xr);
    if (halo) pull(hs, hl, hc, hr);
  };
  auto staged_sum = [&](const T* st, int s) {
    return ((st[0 * SW + s] + st[1 * SW + s]) + (st[2 * SW + s] + st[3 * SW + s])) +
           ((st[4 * SW + s] + st[5 * SW + s]) + (st[6 * SW + s] + st[7 * SW + s])) +
           st[8 * SW + s];
  };
  // mu of logical row r at slots 1 .. w+2 (own slot; threads 0 and 1 also
  // take slots 1 and w+2).
  auto put_mu = [&](int r) {
    const T* rn = rho_s + ((r + 1) & (kRing - 1)) * SW;  // row above (y+1)
    const T* rc = rho_s + (r & (kRing - 1)) * SW;
    const T* rsb = rho_s + ((r - 1) & (kRing - 1)) * SW; // row below (y-1)
    T* mrow = mu_s + (r & (kRing - 1)) * SW;
    auto at = [&](int s) {
      return chem_pot<T>(rc[s], rc[s + 1], rc[s - 1], rn[s], rsb[s], rn[s + 1],
                         rn[s - 1], rsb[s + 1], rsb[s - 1], two_beta, dl, dg, kappa);
    };
    if (own) mrow[sx] = at(sx);
    if (tx == 0) mrow[1] = at(1);
    if (tx == 1) mrow[w + 2] = at(w + 2);
  };

  double st_mass = 0.0, st_kin = 0.0, st_u2 = 0.0;
  double st_mumin = 1e300, st_mumax = -1e300;
  int st_bad = 0;

  const int kfirst = y0 - kHalo, klast = y1 + 1;
  for (int r = kfirst; r < kfirst + PD; ++r) {
    if (r <= klast) request(r);
    cp_async_commit();
  }
  for (int k = kfirst; k <= klast; ++k) {
    if (k + PD <= klast) request(k + PD);
    cp_async_commit();                     // one group per row, possibly empty
    cp_async_wait<PD>();                   // row k has landed (this thread)
    {
      const T* st = stage + (k & (kStages - 1)) * 9 * SW;
      T* row = rho_s + (k & (kRing - 1)) * SW;
      if (own) row[sx] = staged_sum(st, sx);
      if (halo) row[hs] = staged_sum(st, hs);
    }
    __syncthreads();
    if (k - 1 >= y0 - 1) put_mu(k - 1);
    __syncthreads();
    const int c = k - 2;                   // row to collide
    if (c >= y0 && own) {
      const T* r_dn = rho_s + ((c - 1) & (kRing - 1)) * SW;
      const T* r_c = rho_s + (c & (kRing - 1)) * SW;
      const T* r_up = rho_s + ((c + 1) & (kRing - 1)) * SW;
      const T* m_dn = mu_s + ((c - 1) & (kRing - 1)) * SW;
      const T* m_c = mu_s + (c & (kRing - 1)) * SW;
      const T* m_up = mu_s + ((c + 1) & (kRing - 1)) * SW;
      // grad(phi) = (E - W)/3 + (NE + SE - NW - SW)/12, likewise in y
      const T gmx = T(1.0 / 3.0) * (m_c[sx + 1] - m_c[sx - 1]) +
                    T(1.0 / 12.0) * ((m_up[sx + 1] + m_dn[sx + 1]) -
                                     (m_up[sx - 1] + m_dn[sx - 1]));
      const T gmy = T(1.0 / 3.0) * (m_up[sx] - m_dn[sx]) +
                    T(1.0 / 12.0) * ((m_up[sx + 1] + m_up[sx - 1]) -
                                     (m_dn[sx + 1] + m_dn[sx - 1]));
      const T grx = T(1.0 / 3.0) * (r_c[sx + 1] - r_c[sx - 1]) +
                    T(1.0 / 12.0) * ((r_up[sx + 1] + r_dn[sx + 1]) -
                                     (r_up[sx - 1] + r_dn[sx - 1]));
      const T gry = T(1.0 / 3.0) * (r_up[sx] - r_dn[sx]) +
                    T(1.0 / 12.0) * ((r_up[sx + 1] + r_up[sx - 1]) -
                                     (r_dn[sx + 1] + r_dn[sx - 1]));
      const T rs = r_c[sx];
      const T* st = stage + (c & (kStages - 1)) * 9 * SW;
      T g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = st[i * SW + sx];
      T ux, uy;
      collide<T, WB>(g, rs, gmx, gmy, grx, gry, p, ux, uy);
      if (!MOMENTS) {
        const long long o = (long long)c * p.pitch + xc;
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[i * p.plane + o] = g[i];
      } else {
        const double rho = (double)rs + p.rho_ref;
        const double mu = (double)m_c[sx];
        const double dux = (double)ux, duy = (double)uy;
        const long long kk = (long long)c * p.nx + xc;
        if (mo.rho) mo.rho[kk] = rho;
        if (mo.ux) mo.ux[kk] = dux;
        if (mo.uy) mo.uy[kk] = duy;
        if (mo.mu) mo.mu[kk] = mu;
        const double u2 = dux * dux + duy * duy;
        st_mass += rho;
        st_kin += 0.5 * rho * u2;
        st_u2 = fmax(st_u2, u2);
        st_mumin = fmin(st_mumin, mu);
        st_mumax = fmax(st_mumax, mu);
        if (!isfinite(rho) || !isfinite(mu) || !isfinite(u2)) st_bad = 1;
      }
    }
  }
  cp_async_wait<0>();

  if (MOMENTS && mo.partials) {
    // deterministic block reduction: warp shuffle, then thread 0 over warps
    __shared__ double red[kMaxTile / 32][kStatRec];
    double v[kStatRec] = {st_mass, st_kin, st_u2, st_mumin, st_mumax, (double)st_bad};
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
      double* out = mo.partials + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kStatRec;
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) out[q] = r[q];
    }
  }
}

// Final reduction of the per-CTA records, one block, fixed order.
// out: mass, kinetic, umax, mu_min, mu_max, nonfinite.
__global__ void __launch_bounds__(256)
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
__constant__ int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

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
