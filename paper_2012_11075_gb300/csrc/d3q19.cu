// The three-dimensional form of the well-balanced LBE (and of the standard
// LBE) on the D3Q19 lattice, in FP64 or FP32-shifted storage: the wblbe3_*
// part of include/wblbe.h.
//
// The paper builds the well-balanced scheme in D dimensions (Sec. III): the
// equilibrium of Eq. mFeq, F = -rho grad(mu) (Eq. mF) and the forcing term of
// Eq. mFi, whose isotropic term carries D; Sec. V notes the construction
// carries over to other lattice Boltzmann models.  Here D = 3 on D3Q19
// (c_0 = 0; six axis vectors, w = 1/18; twelve edge vectors, w = 1/36;
// w_0 = 1/3; cs^2 = 1/3), with the isotropic central stencils
// grad(phi) = 3 sum_i w_i c_i phi(x + c_i) and
// lap(phi) = 6 sum_i w_i (phi(x + c_i) - phi(x)).
//
// One step is three kernels on the caller's stream (in FP64 the FP64 pipe is
// the limit, not memory traffic; in FP32 the traffic is):
//   d3_density:   rho(x) = sum_i P_i(x - c_i)           (pull, Eq. rhoU)
//   d3_chem_pot:  mu = mu_0(rho) - kappa lap(rho)        (Sec. II)
//   d3_collide:   the pulled populations, grad rho and grad mu, the force,
//                 u, the equilibrium and forcing terms, and the BGK update
//                 (Eq. D2Q9), stored at x for the next pull.
// Layout: nineteen planes P_i[(z ny + y) pitch + x], pitch = nx rounded up
// to 16 elements, two buffers (ping-pong); the planes hold f_i - s_i, with
// s_i the well-balanced rho0 vector s_0 = -(1 - w_0) rho0, s_i = w_i rho0 (0
// for the standard scheme), plus in FP32 the scheme's rest equilibrium at
// rho_ref = rho_g; the update carries the shift unchanged.  The density and
// chemical-potential fields hold rho - rho_ref and mu in the storage type.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>

#include "../../include/wblbe.h"
#include "lbm_kernels.cuh"

using namespace wblbe;

namespace {

constexpr int kQ3 = 19;
constexpr int kBlock3 = 128;
constexpr size_t kAlign3 = 256;

// D3Q19 in the order rest, 6 axis (+x, -x, +y, -y, +z, -z), 12 edges in
// opposite pairs ((1,1,0), (-1,-1,0)), ((1,-1,0), (-1,1,0)), ((1,0,1),
// (-1,0,-1)), ((1,0,-1), (-1,0,1)), ((0,1,1), (0,-1,-1)), ((0,1,-1), (0,-1,1)).
__host__ __device__ constexpr int cx3(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)
             ? 1 : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
}
__host__ __device__ constexpr int cy3(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)
             ? 1 : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
}
__host__ __device__ constexpr int cz3(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)
             ? 1 : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
}
__host__ __device__ constexpr double w3(int i) {
  return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
}

struct P3 {
  int nx, ny, nz, pitch;
  long long plane;                 // elements per population plane / field
  double omega, kforce, kappa, two_beta, rho_l, rho_g;
  // storage shift density (0 in FP64) and rho_ref - rho_l, rho_ref - rho_g
  double rho_ref, dl, dg;
  long long step;                  // the step being taken (FP32 rounding draws)
};

// Mirror-symmetric sum of the eighteen moving populations: opposite pairs
// first, the axis pairs together and the edge pairs by plane, so that a
// reflection of any axis maps the grouping onto itself (mirror-image nodes
// round alike; the FP32 path).
template <typename T>
__device__ __forceinline__ T moving_sum3(const T (&g)[19]) {
  const T ax = ((g[1] + g[2]) + (g[3] + g[4])) + (g[5] + g[6]);
  const T xy = (g[7] + g[8]) + (g[9] + g[10]);
  const T xz = (g[11] + g[12]) + (g[13] + g[14]);
  const T yz = (g[15] + g[16]) + (g[17] + g[18]);
  return ax + ((xy + xz) + yz);
}

// Single-node forms of the FP32 exact-mass rounding of the 2D kernel:
// TwoSum (Knuth), a uniform draw in [0, 1) on a 2^-23 grid from the node key
// k and the step key ht (MurmurHash3's finalizer), and the stochastic
// rounding of h + e to h or its neighbour on the side of e with probability
// |e| / gap.
__device__ __forceinline__ void two_sum1(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}
__device__ __forceinline__ float node_uniform(uint32_t k, uint32_t ht) {
  return __fsub_rn(__uint_as_float(0x3f800000u | (fmix32(k + ht) >> 9)), 1.0f);
}
__device__ __forceinline__ float round_stochastic1(float h, float e, float u) {
  const float n = next_toward(h, e);
  return fabsf(__fmul_rn(u, __fsub_rn(n, h))) < fabsf(e) ? n : h;
}

struct Out3 {
  double* rho;                     // [nz][ny][nx] fields (may be null)
  double* ux;
  double* uy;
  double* uz;
  double* mu;
  double* partials;                // per-block stats records (may be null)
};

__device__ __forceinline__ int wrap3(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ long long at3(const P3& p, int x, int y, int z) {
  return ((long long)z * p.ny + y) * p.pitch + x;
}

// rho = sum_i f_i with f_i(x) = P_i(x - c_i): in FP64 summed from i = 0 to
// 18; in FP32 the stored deviation rs = rho - rho_ref = g_0 + the
// mirror-symmetric moving sum (the collision repeats that sum for the exact
// mass balance).
template <typename T>
__global__ void __launch_bounds__(kBlock3) d3_density(const T* __restrict__ src,
                                                      T* __restrict__ rho, const P3 p) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  if (sizeof(T) == 8) {
    T s = src[at3(p, x, y, z)];                   // f_0 (c_0 = 0)
#pragma unroll
    for (int i = 1; i < kQ3; ++i)
      s += src[i * p.plane + at3(p, wrap3(x - cx3(i), p.nx), wrap3(y - cy3(i), p.ny),
                                 wrap3(z - cz3(i), p.nz))];
    rho[at3(p, x, y, z)] = s;
  } else {
    T g[kQ3];
#pragma unroll
    for (int i = 0; i < kQ3; ++i)
      g[i] = src[i * p.plane + at3(p, wrap3(x - cx3(i), p.nx), wrap3(y - cy3(i), p.ny),
                                   wrap3(z - cz3(i), p.nz))];
    rho[at3(p, x, y, z)] = g[0] + moving_sum3(g);
  }
}

// mu = mu_0(rho) - kappa lap(rho), mu_0 = 2 beta a b (a + b), a = rho - rho_l,
// b = rho - rho_g (Eq. doubleWell), lap = 6 sum_i w_i (rho(x + c_i) - rho(x)).
// The field holds rho - rho_ref (rho_ref = 0 in FP64), which the Laplacian
// does not see and a, b take up through dl = rho_ref - rho_l, dg.
template <typename T>
__global__ void __launch_bounds__(kBlock3) d3_chem_pot(const T* __restrict__ rho,
                                                       T* __restrict__ mu, const P3 p) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  const T c = rho[at3(p, x, y, z)];
  // sums of the axis and edge neighbours, then the centre's share taken off
  // once per sum (rather than from every neighbour): 6 (ax/18 + ed/36)
  auto nbr = [&](int i) {
    return __ldg(rho + at3(p, wrap3(x + cx3(i), p.nx), wrap3(y + cy3(i), p.ny),
                           wrap3(z + cz3(i), p.nz)));
  };
  T ax = nbr(1), ed = nbr(7);
#pragma unroll
  for (int i = 2; i < kQ3; ++i) {
    if (i == 7) continue;
    if (i < 7) ax += nbr(i); else ed += nbr(i);
  }
  const T lap = T(1.0 / 3.0) * (ax - T(6) * c) + T(1.0 / 6.0) * (ed - T(12) * c);
  const T a = c + T(p.dl), b = c + T(p.dg);
  mu[at3(p, x, y, z)] = T(p.two_beta) * a * b * (a + b) - T(p.kappa) * lap;
}

// 12 grad(phi) = 36 sum_i w_i c_i phi(x + c_i): 2 (axis differences) +
// (edge differences); the factor 1/12 is folded into the constants that
// use the gradients.
template <typename T>
__device__ __forceinline__ void grad3x12(const T* __restrict__ phi, const P3& p, int x, int y,
                                         int z, T& gx, T& gy, T& gz) {
  auto v = [&](int dx, int dy, int dz) {
    return __ldg(phi + at3(p, wrap3(x + dx, p.nx), wrap3(y + dy, p.ny), wrap3(z + dz, p.nz)));
  };
  const T axx = v(1, 0, 0) - v(-1, 0, 0), axy = v(0, 1, 0) - v(0, -1, 0),
          axz = v(0, 0, 1) - v(0, 0, -1);
  const T exy1 = v(1, 1, 0) - v(-1, -1, 0), exy2 = v(1, -1, 0) - v(-1, 1, 0);
  const T exz1 = v(1, 0, 1) - v(-1, 0, -1), exz2 = v(1, 0, -1) - v(-1, 0, 1);
  const T eyz1 = v(0, 1, 1) - v(0, -1, -1), eyz2 = v(0, 1, -1) - v(0, -1, 1);
  gx = T(2) * axx + ((exy1 + exy2) + (exz1 + exz2));
  gy = T(2) * axy + ((exy1 - exy2) + (eyz1 + eyz2));
  gz = T(2) * axz + ((exz1 - exz2) + (eyz1 - eyz2));
}

// The collision of one node, and its stores (MOMENTS: fields and stats
// instead).  For an opposite pair (i, i') the even part E and the odd part
// O of omega f^eq + kforce F_i are shared, g_i' = keep g_i + E + O,
// g_i'' = keep g_i' + E - O, with
//   E = w (t + cu (omega rho 9/2 cu + 9 kforce cG) + kforce h (u.grad rho))
//       [+ omega w rho for the standard equilibrium],
//   O = 3 w (omega rho cu + kforce cF),
//   t = -3/2 omega rho u.u - 3 kforce u.G,
// G = F + cs^2 grad rho and h = (3|c|^2 - 3)/2 (Eq. mFi, D = 3) for the
// well-balanced scheme, G = F and h = 0 for the standard one (Eq. Fi).
template <typename T, bool WB, bool MOMENTS>
__global__ void __launch_bounds__(kBlock3) d3_collide(const T* __restrict__ src,
                                                      T* __restrict__ dst,
                                                      const T* __restrict__ rho,
                                                      const T* __restrict__ mu,
                                                      const P3 p, const Out3 out) {
  constexpr bool kShifted = sizeof(T) == 4;    // FP32 stores g_i = f_i - s_i
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  const bool own = x < p.nx;
  double st[kStatRec] = {0.0, 0.0, 0.0, 1e300, -1e300, 0.0};
  if (own) {
    T g[kQ3];
#pragma unroll
    for (int i = 0; i < kQ3; ++i)
      g[i] = src[i * p.plane + at3(p, wrap3(x - cx3(i), p.nx), wrap3(y - cy3(i), p.ny),
                                   wrap3(z - cz3(i), p.nz))];
    const long long k = at3(p, x, y, z);
    const T rs = rho[k];                         // rho - rho_ref (rho in FP64)
    const T r = kShifted ? rs + T(p.rho_ref) : rs;
    // 12 grad mu, 12 grad rho; F = -rho grad mu (Eq. mF), or the potential
    // form cs^2 grad rho - rho grad mu of the standard scheme
    T gmx, gmy, gmz, grx, gry, grz;
    grad3x12<T>(mu, p, x, y, z, gmx, gmy, gmz);
    grad3x12<T>(rho, p, x, y, z, grx, gry, grz);
    const T nr = r * T(-1.0 / 12.0);
    T Fx, Fy, Fz;
    if (WB) {
      Fx = nr * gmx;
      Fy = nr * gmy;
      Fz = nr * gmz;
    } else {
      Fx = T(1.0 / 36.0) * grx + nr * gmx;
      Fy = T(1.0 / 36.0) * gry + nr * gmy;
      Fz = T(1.0 / 36.0) * grz + nr * gmz;
    }
    // momentum from the differences of opposite pairs (each edge difference
    // serves two components)
    const T d12 = g[1] - g[2], d34 = g[3] - g[4], d56 = g[5] - g[6];
    const T d78 = g[7] - g[8], d910 = g[9] - g[10], d1112 = g[11] - g[12];
    const T d1314 = g[13] - g[14], d1516 = g[15] - g[16], d1718 = g[17] - g[18];
    const T jx = ((d12 + d78) + (d910 + d1112)) + d1314;
    const T jy = ((d34 + d78) - (d910 - d1516)) + d1718;
    const T jz = ((d56 + d1112) - (d1314 - d1516)) - d1718;
    const T inv = recip(r);
    const T ux = (jx + T(0.5) * Fx) * inv, uy = (jy + T(0.5) * Fy) * inv,
            uz = (jz + T(0.5) * Fz) * inv;                       // Eq. rhoU
    const T muc = mu[k];
    if (MOMENTS) {
      const double rd = kShifted ? (double)rs + p.rho_ref : (double)r;
      const double uxd = ux, uyd = uy, uzd = uz, mud = muc;
      if (out.rho) out.rho[(size_t)(z * p.ny + y) * p.nx + x] = rd;
      if (out.ux) out.ux[(size_t)(z * p.ny + y) * p.nx + x] = uxd;
      if (out.uy) out.uy[(size_t)(z * p.ny + y) * p.nx + x] = uyd;
      if (out.uz) out.uz[(size_t)(z * p.ny + y) * p.nx + x] = uzd;
      if (out.mu) out.mu[(size_t)(z * p.ny + y) * p.nx + x] = mud;
      const double u2 = uxd * uxd + uyd * uyd + uzd * uzd;
      st[0] = rd;
      st[1] = 0.5 * rd * u2;
      st[2] = u2;
      st[3] = mud;
      st[4] = mud;
      st[5] = (!isfinite(rd) || !isfinite(mud) || !isfinite(u2)) ? 1.0 : 0.0;
    } else {
      T om = T(p.omega);
      const T kf = T(p.kforce);
      T keep = T(1) - om;
      if (kShifted && om < T(0.5)) {
        // keep + omega == 1 exactly in float (the update then conserves
        // mass); 1 - omega is exact by Sterbenz only for omega >= 1/2
        keep = T(1.0 - p.omega);
        om = T(1) - keep;
      }
      // FP32: the moving populations' sum before the collision (the same
      // grouping as the density), for the exact node mass balance below
      const T m_in = kShifted ? moving_sum3(g) : T(0);
      T Gx = Fx, Gy = Fy, Gz = Fz;
      if (WB) {
        Gx = Fx + T(1.0 / 36.0) * grx;                          // G = F + cs^2 grad rho
        Gy = Fy + T(1.0 / 36.0) * gry;
        Gz = Fz + T(1.0 / 36.0) * grz;
      }
      const T orho = om * r;
      const T obase = om * rs;                   // omega (rho - rho_ref): the stored base
      const T t = T(-1.5) * orho * (ux * ux + uy * uy + uz * uz) -
                  T(3.0) * kf * (ux * Gx + uy * Gy + uz * Gz);
      const T ku = WB ? (kf * T(1.0 / 12.0)) * (ux * grx + uy * gry + uz * grz) : T(0);
      // per-node constants of the pairs, with the weights folded in
      // (w_ax = 1/18, w_edge = 1/36): E = C + cu (A cu + K.c), O = 3 w c.M
      const T Ca = WB ? T(1.0 / 18.0) * t : T(1.0 / 18.0) * (t + obase);
      const T Ce = WB ? T(1.0 / 36.0) * (t + T(1.5) * ku) : T(1.0 / 36.0) * (t + obase);
      const T Aa = T(0.25) * orho, Ae = T(0.125) * orho;         // w 9/2 omega rho
      const T kh = T(0.5) * kf, kq = T(0.25) * kf, k6 = kf * T(1.0 / 6.0);
      const T Kax = kh * Gx, Kay = kh * Gy, Kaz = kh * Gz;       // 9 w_ax kforce G
      const T Kex = kq * Gx, Key = kq * Gy, Kez = kq * Gz;       // 9 w_edge kforce G
      const T o6 = orho * T(1.0 / 6.0);                          // 3 w_ax (omega rho u + kforce F)
      const T Mx = o6 * ux + k6 * Fx, My = o6 * uy + k6 * Fy, Mz = o6 * uz + k6 * Fz;
      auto axis = [&](int i, int j, T cu, T K, T M) {
        const T E = Ca + cu * (Aa * cu + K);
        g[i] = keep * g[i] + (E + M);
        g[j] = keep * g[j] + (E - M);
        return E;
      };
      // edge pair: 3 w_edge c.M = (Ma + Mb) / 2 for c = a + b
      auto edge = [&](int i, int j, T cu, T K, T S) {
        const T E = Ce + cu * (Ae * cu + K);
        g[i] = keep * g[i] + (E + T(0.5) * S);
        g[j] = keep * g[j] + (E - T(0.5) * S);
        return E;
      };
      const T Ea1 = axis(1, 2, ux, Kax, Mx);
      const T Ea2 = axis(3, 4, uy, Kay, My);
      const T Ea3 = axis(5, 6, uz, Kaz, Mz);
      const T Ee1 = edge(7, 8, ux + uy, Kex + Key, Mx + My);
      const T Ee2 = edge(9, 10, ux - uy, Kex - Key, Mx - My);
      const T Ee3 = edge(11, 12, ux + uz, Kex + Kez, Mx + Mz);
      const T Ee4 = edge(13, 14, ux - uz, Kex - Kez, Mx - Mz);
      const T Ee5 = edge(15, 16, uy + uz, Key + Kez, My + Mz);
      const T Ee6 = edge(17, 18, uy - uz, Key - Kez, My - Mz);
      if constexpr (kShifted) {
        if (WB) {
          // The collision conserves the node's mass, so the rest population
          // follows from the balance: g_0' = g_0 + omega m_in - 2 sum E (the
          // moving ones leave as keep g + E +- O).  Its small one-signed
          // O(u^2) part would be lost in rounding g_0 ~ rho - rho_ref to
          // float; TwoSum keeps the remainder and a zero-mean rounding,
          // seeded by the node and the step, takes it into account.
          const T sE = ((Ea1 + Ea2) + Ea3) + (((Ee1 + Ee2) + (Ee3 + Ee4)) + (Ee5 + Ee6));
          T hsum, err;
          two_sum1(g[0], __fmaf_rn(-2.0f, sE, om * m_in), hsum, err);
          const uint32_t key = (uint32_t)(((long long)z * p.ny + y) * p.nx + x);
          g[0] = round_stochastic1(hsum, err, node_uniform(key, step_key(p.step)));
        } else {
          g[0] = rs - moving_sum3(g);          // the standard scheme: the mass balance
        }
      } else {
        (void)Ea1; (void)Ea2; (void)Ea3; (void)Ee1; (void)Ee2; (void)Ee3;
        (void)Ee4; (void)Ee5; (void)Ee6; (void)m_in;
        // rest: WB f_0^eq - s_0 = rho - w_0 3/2 rho u.u, F_0 = w_0 (-3 u.G - 3/2 u.grad rho);
        // standard f_0^eq = w_0 rho (1 - 3/2 u.u), F_0 = w_0 (-3 u.G)
        const T w0 = T(1.0 / 3.0);
        g[0] = keep * g[0] + (WB ? obase + w0 * (t - T(1.5) * ku) : w0 * (t + obase));
      }
#pragma unroll
      for (int i = 0; i < kQ3; ++i) dst[i * p.plane + k] = g[i];
    }
  }
  if (MOMENTS && out.partials) {
    __shared__ double red[kBlock3 / 32][kStatRec];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o0 = __shfl_down_sync(0xffffffffu, st[0], off);
      const double o1 = __shfl_down_sync(0xffffffffu, st[1], off);
      const double o2 = __shfl_down_sync(0xffffffffu, st[2], off);
      const double o3 = __shfl_down_sync(0xffffffffu, st[3], off);
      const double o4 = __shfl_down_sync(0xffffffffu, st[4], off);
      const double o5 = __shfl_down_sync(0xffffffffu, st[5], off);
      st[0] += o0;
      st[1] += o1;
      st[2] = fmax(st[2], o2);
      st[3] = fmin(st[3], o3);
      st[4] = fmax(st[4], o4);
      st[5] = fmax(st[5], o5);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) red[warp][q] = st[q];
    __syncthreads();
    if (threadIdx.x == 0) {
      double r[kStatRec];
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) r[q] = red[0][q];
      for (int w = 1; w < kBlock3 / 32; ++w) {
        r[0] += red[w][0];
        r[1] += red[w][1];
        r[2] = fmax(r[2], red[w][2]);
        r[3] = fmin(r[3], red[w][3]);
        r[4] = fmax(r[4], red[w][4]);
        r[5] = fmax(r[5], red[w][5]);
      }
      double* o = out.partials +
                  (size_t)((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * kStatRec;
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) o[q] = r[q];
    }
  }
}

// f = f^eq(rho, 0) stored for the pull: P_i(x) = f_i^eq(rho(x + c_i)) - s_i.
template <typename T>
__global__ void d3_init(const double* __restrict__ rho_in, T* __restrict__ dst, const P3 p,
                        int wb) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
#pragma unroll
  for (int i = 0; i < kQ3; ++i) {
    const int xx = wrap3(x + cx3(i), p.nx), yy = wrap3(y + cy3(i), p.ny),
              zz = wrap3(z + cz3(i), p.nz);
    const double r = rho_in[(size_t)(zz * p.ny + yy) * p.nx + xx] - p.rho_ref;
    // WB: f_0^eq - s_0 = rho - rho_ref, f_i^eq - s_i = 0; standard: w_i (rho - rho_ref)
    dst[i * p.plane + at3(p, x, y, z)] = (T)(wb ? (i == 0 ? r : 0.0) : w3(i) * r);
  }
}

// f_i(x) = P_i(x - c_i) + s_i for one direction, [nz][ny][nx].
template <typename T>
__global__ void d3_get(const T* __restrict__ src, double* __restrict__ f, const P3 p, int dir,
                       double shift) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  const double v = (double)src[dir * p.plane + at3(p, wrap3(x - cx3(dir), p.nx),
                                                   wrap3(y - cy3(dir), p.ny),
                                                   wrap3(z - cz3(dir), p.nz))];
  f[(size_t)(z * p.ny + y) * p.nx + x] = v + shift;
}

thread_local char g_d3_error[256] = "";

size_t align3(size_t v) { return (v + kAlign3 - 1) / kAlign3 * kAlign3; }

struct Layout3 {
  int pitch;
  long long plane;
  size_t off_a, off_b, off_rho, off_mu, off_stage, off_partials, off_stats, total;
  long long records;
};

size_t elem3(const wblbe3_params* p) { return p->precision == WBLBE_FP64 ? 8 : 4; }

Layout3 layout3(const wblbe3_params* p) {
  Layout3 L{};
  L.pitch = (p->nx + 15) / 16 * 16;
  L.plane = (long long)L.pitch * p->ny * p->nz;
  const size_t pops = align3((size_t)kQ3 * L.plane * elem3(p));
  const size_t field = align3((size_t)L.plane * elem3(p));
  L.records = (long long)((p->nx + kBlock3 - 1) / kBlock3) * p->ny * p->nz;
  size_t off = 0;
  L.off_a = off; off += pops;
  L.off_b = off; off += pops;
  L.off_rho = off; off += field;
  L.off_mu = off; off += field;
  L.off_stage = off; off += align3((size_t)p->nx * p->ny * p->nz * sizeof(double));
  L.off_partials = off; off += align3((size_t)L.records * kStatRec * sizeof(double));
  L.off_stats = off; off += align3(8 * sizeof(double));
  L.total = off;
  return L;
}

bool params3_valid(const wblbe3_params* p, char* why, size_t n) {
  if (!p) { snprintf(why, n, "params is NULL"); return false; }
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) { snprintf(why, n, "nx, ny, nz must be >= 1"); return false; }
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) { snprintf(why, n, "tau must be > 0.5"); return false; }
  if (!(p->kappa >= 0.0) || !(p->beta > 0.0)) { snprintf(why, n, "need kappa >= 0, beta > 0"); return false; }
  if (!(p->rho_g > 0.0) || !(p->rho_l > p->rho_g)) { snprintf(why, n, "need rho_l > rho_g > 0"); return false; }
  if (!std::isfinite(p->rho0)) { snprintf(why, n, "rho0 must be finite"); return false; }
  if (p->scheme != WBLBE_STANDARD && p->scheme != WBLBE_WELL_BALANCED) {
    snprintf(why, n, "the D3Q19 path runs the standard and well-balanced schemes"); return false;
  }
  if (p->precision != WBLBE_FP64 && p->precision != WBLBE_FP32_SHIFTED) {
    snprintf(why, n, "unknown precision %d", p->precision); return false;
  }
  if ((long long)((p->nx + 15) / 16 * 16) * p->ny * p->nz >= (1LL << 40) ||
      p->ny > 65535 || p->nz > 65535) {
    snprintf(why, n, "lattice too large (ny, nz <= 65535)"); return false;
  }
  return true;
}

}  // namespace

struct wblbe3_ctx {
  wblbe3_params p;
  Layout3 L;
  int device;
  cudaStream_t stream;
  void* buf[2];                   // population buffers (float64 or float32)
  int cur;
  void *rho, *mu;                 // rho - rho_ref and mu fields (the same type)
  double *stage, *partials, *stats;
  int64_t steps, launches;
  double mass0;
  bool have_state;
  char err[256];
};

namespace {

wblbe_status f3(wblbe3_ctx* h, wblbe_status st, const char* fmt, ...) {
  char* dst = h ? h->err : g_d3_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 256, fmt, ap);
  va_end(ap);
  return st;
}

#define CU3(h, call)                                                         \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return f3((h), WBLBE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
  } while (0)

P3 p3_of(const wblbe3_ctx* h) {
  P3 q{};
  q.nx = h->p.nx;
  q.ny = h->p.ny;
  q.nz = h->p.nz;
  q.pitch = h->L.pitch;
  q.plane = h->L.plane;
  q.omega = 1.0 / h->p.tau;
  q.kforce = 1.0 - 1.0 / (2.0 * h->p.tau);
  q.kappa = h->p.kappa;
  q.two_beta = 2.0 * h->p.beta;
  q.rho_l = h->p.rho_l;
  q.rho_g = h->p.rho_g;
  // FP32 stores deviations from the rest equilibrium at rho_ref = rho_g
  q.rho_ref = h->p.precision == WBLBE_FP64 ? 0.0 : h->p.rho_g;
  q.dl = q.rho_ref - h->p.rho_l;
  q.dg = q.rho_ref - h->p.rho_g;
  q.step = h->steps;
  return q;
}

dim3 grid3(const wblbe3_ctx* h) {
  return dim3((h->p.nx + kBlock3 - 1) / kBlock3, h->p.ny, h->p.nz);
}

// The stored shift s_i: the well-balanced rho0 vector, plus in FP32 the
// scheme's rest equilibrium at rho_ref = rho_g.
double shift3(const wblbe3_params& p, int i) {
  const double rr = p.precision == WBLBE_FP64 ? 0.0 : p.rho_g;
  if (p.scheme != WBLBE_WELL_BALANCED) return w3(i) * rr;
  return i == 0 ? rr - (1.0 - w3(0)) * p.rho0 : w3(i) * p.rho0;
}

// density and chemical potential of the current state, then the collision
// (step: into the other buffer) or the moments (fields and stats).
template <typename T>
void pass3_typed(wblbe3_ctx* h, bool moments, const Out3& out, const P3& q, dim3 g) {
  const T* src = static_cast<const T*>(h->buf[h->cur]);
  T* dst = static_cast<T*>(h->buf[1 - h->cur]);
  T* rho = static_cast<T*>(h->rho);
  T* mu = static_cast<T*>(h->mu);
  d3_density<T><<<g, kBlock3, 0, h->stream>>>(src, rho, q);
  d3_chem_pot<T><<<g, kBlock3, 0, h->stream>>>(rho, mu, q);
  const bool wb = h->p.scheme == WBLBE_WELL_BALANCED;
  if (moments) {
    if (wb) d3_collide<T, true, true><<<g, kBlock3, 0, h->stream>>>(src, nullptr, rho, mu, q, out);
    else d3_collide<T, false, true><<<g, kBlock3, 0, h->stream>>>(src, nullptr, rho, mu, q, out);
  } else {
    if (wb) d3_collide<T, true, false><<<g, kBlock3, 0, h->stream>>>(src, dst, rho, mu, q, out);
    else d3_collide<T, false, false><<<g, kBlock3, 0, h->stream>>>(src, dst, rho, mu, q, out);
  }
}

wblbe_status pass3(wblbe3_ctx* h, bool moments, const Out3& out) {
  const P3 q = p3_of(h);
  const dim3 g = grid3(h);
  if (h->p.precision == WBLBE_FP64)
    pass3_typed<double>(h, moments, out, q, g);
  else
    pass3_typed<float>(h, moments, out, q, g);
  CU3(h, cudaGetLastError());
  h->launches += 3;
  return WBLBE_OK;
}

wblbe_status stats3(wblbe3_ctx* h, double* rho, double* ux, double* uy, double* uz, double* mu,
                    wblbe_stats* st) {
  Out3 out{rho, ux, uy, uz, mu, h->partials};
  wblbe_status s = pass3(h, true, out);
  if (s != WBLBE_OK) return s;
  stats_finalize_kernel<<<1, 256, 0, h->stream>>>(h->partials, (int)h->L.records, h->stats);
  CU3(h, cudaGetLastError());
  h->launches += 1;
  double v[kStatRec];
  CU3(h, cudaMemcpyAsync(v, h->stats, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  CU3(h, cudaStreamSynchronize(h->stream));
  if (st) {
    st->step = h->steps;
    st->mass = v[0];
    st->kinetic = v[1];
    st->umax = v[2];
    st->mu_min = v[3];
    st->mu_max = v[4];
    st->nonfinite = v[5] != 0.0 || !std::isfinite(v[0]);
    st->mass_drift_rel = h->mass0 != 0.0 ? (v[0] - h->mass0) / h->mass0 : 0.0;
  }
  return WBLBE_OK;
}

}  // namespace

extern "C" {

size_t wblbe3_workspace_bytes(const wblbe3_params* params) {
  char why[256];
  if (!params3_valid(params, why, sizeof(why))) return 0;
  return layout3(params).total;
}

wblbe_status wblbe3_create(const wblbe3_params* params, void* dev_workspace,
                           size_t workspace_bytes, void* cuda_stream, wblbe3_handle* out) {
  char why[256];
  if (!out) return f3(nullptr, WBLBE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params3_valid(params, why, sizeof(why))) return f3(nullptr, WBLBE_EINVAL, "%s", why);
  const Layout3 L = layout3(params);
  if (!dev_workspace || ((uintptr_t)dev_workspace % kAlign3) != 0)
    return f3(nullptr, WBLBE_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < L.total)
    return f3(nullptr, WBLBE_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, L.total);
  if (L.records > 0x7fffffffLL) return f3(nullptr, WBLBE_EINVAL, "lattice too large");
  wblbe3_ctx* h = new (std::nothrow) wblbe3_ctx();
  if (!h) return f3(nullptr, WBLBE_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return f3(nullptr, WBLBE_ECUDA, "no CUDA device");
  }
  unsigned char* ws = static_cast<unsigned char*>(dev_workspace);
  h->p = *params;
  h->L = L;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->buf[0] = ws + L.off_a;
  h->buf[1] = ws + L.off_b;
  h->rho = ws + L.off_rho;
  h->mu = ws + L.off_mu;
  h->stage = reinterpret_cast<double*>(ws + L.off_stage);
  h->partials = reinterpret_cast<double*>(ws + L.off_partials);
  h->stats = reinterpret_cast<double*>(ws + L.off_stats);
  *out = h;
  return WBLBE_OK;
}

wblbe_status wblbe3_init_rho(wblbe3_handle h, const double* rho, int32_t rho_on_device) {
  if (!h) return f3(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!rho) return f3(h, WBLBE_EINVAL, "rho is NULL");
  const double* src = rho;
  if (!rho_on_device) {
    CU3(h, cudaMemcpyAsync(h->stage, rho, (size_t)h->p.nx * h->p.ny * h->p.nz * sizeof(double),
                           cudaMemcpyHostToDevice, h->stream));
    src = h->stage;
  }
  h->cur = 0;
  const int wb = h->p.scheme == WBLBE_WELL_BALANCED;
  if (h->p.precision == WBLBE_FP64)
    d3_init<double><<<grid3(h), kBlock3, 0, h->stream>>>(
        src, static_cast<double*>(h->buf[0]), p3_of(h), wb);
  else
    d3_init<float><<<grid3(h), kBlock3, 0, h->stream>>>(
        src, static_cast<float*>(h->buf[0]), p3_of(h), wb);
  CU3(h, cudaGetLastError());
  h->launches += 1;
  h->steps = 0;
  h->have_state = true;
  wblbe_stats s{};
  wblbe_status st = stats3(h, nullptr, nullptr, nullptr, nullptr, nullptr, &s);
  if (st != WBLBE_OK) return st;
  h->mass0 = s.mass;
  return WBLBE_OK;
}

wblbe_status wblbe3_step(wblbe3_handle h, int64_t nsteps) {
  if (!h) return f3(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (nsteps < 0) return f3(h, WBLBE_EINVAL, "nsteps must be >= 0");
  if (!h->have_state) return f3(h, WBLBE_EINVAL, "no state: call wblbe3_init_rho first");
  for (int64_t n = 0; n < nsteps; ++n) {
    wblbe_status st = pass3(h, false, Out3{});
    if (st != WBLBE_OK) return st;
    h->cur ^= 1;
    h->steps += 1;
  }
  return WBLBE_OK;
}

wblbe_status wblbe3_moments(wblbe3_handle h, double* rho, double* u, double* mu,
                            int32_t out_on_device, wblbe_stats* stats) {
  if (!h) return f3(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!h->have_state) return f3(h, WBLBE_EINVAL, "no state: call wblbe3_init_rho first");
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz;
  if (out_on_device)
    return stats3(h, rho, u, u ? u + n : nullptr, u ? u + 2 * n : nullptr, mu, stats);
  // host outputs: one field at a time through the staging field
  double* outs[5] = {rho, u, u ? u + n : nullptr, u ? u + 2 * n : nullptr, mu};
  bool any = false;
  for (int q = 0; q < 5; ++q) {
    if (!outs[q]) continue;
    any = true;
    double* dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    dev[q] = h->stage;
    wblbe_status st = stats3(h, dev[0], dev[1], dev[2], dev[3], dev[4], stats);
    if (st != WBLBE_OK) return st;
    CU3(h, cudaMemcpyAsync(outs[q], h->stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
  }
  if (!any) return stats3(h, nullptr, nullptr, nullptr, nullptr, nullptr, stats);
  CU3(h, cudaStreamSynchronize(h->stream));
  return WBLBE_OK;
}

wblbe_status wblbe3_get_populations(wblbe3_handle h, double* f, int32_t on_device) {
  if (!h) return f3(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!f) return f3(h, WBLBE_EINVAL, "f is NULL");
  if (!h->have_state) return f3(h, WBLBE_EINVAL, "no state: call wblbe3_init_rho first");
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz;
  for (int i = 0; i < kQ3; ++i) {
    double* dst = on_device ? f + i * n : h->stage;
    if (h->p.precision == WBLBE_FP64)
      d3_get<double><<<grid3(h), kBlock3, 0, h->stream>>>(
          static_cast<const double*>(h->buf[h->cur]), dst, p3_of(h), i, shift3(h->p, i));
    else
      d3_get<float><<<grid3(h), kBlock3, 0, h->stream>>>(
          static_cast<const float*>(h->buf[h->cur]), dst, p3_of(h), i, shift3(h->p, i));
    CU3(h, cudaGetLastError());
    h->launches += 1;
    if (!on_device)
      CU3(h, cudaMemcpyAsync(f + i * n, h->stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
  }
  CU3(h, cudaStreamSynchronize(h->stream));
  return WBLBE_OK;
}

int64_t wblbe3_step_count(wblbe3_handle h) { return h ? h->steps : -1; }
int64_t wblbe3_kernel_launches(wblbe3_handle h) { return h ? h->launches : -1; }

wblbe_status wblbe3_destroy(wblbe3_handle h) {
  if (!h) return f3(nullptr, WBLBE_EINVAL, "handle is NULL");
  cudaStreamSynchronize(h->stream);
  delete h;
  return WBLBE_OK;
}

const char* wblbe3_last_error(wblbe3_handle h) { return h ? h->err : g_d3_error; }

}  // extern "C"
