// The three-dimensional form of the well-balanced LBE (and of the standard
// LBE) on the D3Q19 lattice, FP64: the wblbe3_* half of include/wblbe.h.
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
// One step is three kernels on the caller's stream (FP64 arithmetic is the
// limit here, not memory traffic):
//   d3_density:   rho(x) = sum_i P_i(x - c_i)           (pull, Eq. rhoU)
//   d3_chem_pot:  mu = mu_0(rho) - kappa lap(rho)        (Sec. II)
//   d3_collide:   the pulled populations, grad rho and grad mu, the force,
//                 u, the equilibrium and forcing terms, and the BGK update
//                 (Eq. D2Q9), stored at x for the next pull.
// Layout: nineteen planes P_i[(z ny + y) pitch + x], pitch = nx rounded up
// to 128 bytes, two buffers (ping-pong); the planes hold f_i - s_i with the
// well-balanced rho0 vector s_0 = -(1 - w_0) rho0, s_i = w_i rho0 (0 for the
// standard scheme), which the update carries unchanged.
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
};

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

// rho = sum_i f_i with f_i(x) = P_i(x - c_i), summed from i = 0 to 18.
__global__ void __launch_bounds__(kBlock3) d3_density(const double* __restrict__ src,
                                                      double* __restrict__ rho, const P3 p) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  double s = src[at3(p, x, y, z)];              // f_0 (c_0 = 0)
#pragma unroll
  for (int i = 1; i < kQ3; ++i)
    s += src[i * p.plane + at3(p, wrap3(x - cx3(i), p.nx), wrap3(y - cy3(i), p.ny),
                               wrap3(z - cz3(i), p.nz))];
  rho[at3(p, x, y, z)] = s;
}

// mu = mu_0(rho) - kappa lap(rho), mu_0 = 2 beta a b (a + b), a = rho - rho_l,
// b = rho - rho_g (Eq. doubleWell), lap = 6 sum_i w_i (rho(x + c_i) - rho(x)).
__global__ void __launch_bounds__(kBlock3) d3_chem_pot(const double* __restrict__ rho,
                                                       double* __restrict__ mu, const P3 p) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  const double c = rho[at3(p, x, y, z)];
  // sums of the axis and edge neighbours, then the centre's share taken off
  // once per sum (rather than from every neighbour): 6 (ax/18 + ed/36)
  auto nbr = [&](int i) {
    return __ldg(rho + at3(p, wrap3(x + cx3(i), p.nx), wrap3(y + cy3(i), p.ny),
                           wrap3(z + cz3(i), p.nz)));
  };
  double ax = nbr(1), ed = nbr(7);
#pragma unroll
  for (int i = 2; i < kQ3; ++i) {
    if (i == 7) continue;
    if (i < 7) ax += nbr(i); else ed += nbr(i);
  }
  const double lap = (1.0 / 3.0) * (ax - 6.0 * c) + (1.0 / 6.0) * (ed - 12.0 * c);
  const double a = c - p.rho_l, b = c - p.rho_g;
  mu[at3(p, x, y, z)] = p.two_beta * a * b * (a + b) - p.kappa * lap;
}

// 12 grad(phi) = 36 sum_i w_i c_i phi(x + c_i): 2 (axis differences) +
// (edge differences); the factor 1/12 is folded into the constants that
// use the gradients.
__device__ __forceinline__ void grad3x12(const double* __restrict__ phi, const P3& p, int x,
                                         int y, int z, double& gx, double& gy, double& gz) {
  auto v = [&](int dx, int dy, int dz) {
    return __ldg(phi + at3(p, wrap3(x + dx, p.nx), wrap3(y + dy, p.ny), wrap3(z + dz, p.nz)));
  };
  const double axx = v(1, 0, 0) - v(-1, 0, 0), axy = v(0, 1, 0) - v(0, -1, 0),
               axz = v(0, 0, 1) - v(0, 0, -1);
  const double exy1 = v(1, 1, 0) - v(-1, -1, 0), exy2 = v(1, -1, 0) - v(-1, 1, 0);
  const double exz1 = v(1, 0, 1) - v(-1, 0, -1), exz2 = v(1, 0, -1) - v(-1, 0, 1);
  const double eyz1 = v(0, 1, 1) - v(0, -1, -1), eyz2 = v(0, 1, -1) - v(0, -1, 1);
  gx = 2.0 * axx + ((exy1 + exy2) + (exz1 + exz2));
  gy = 2.0 * axy + ((exy1 - exy2) + (eyz1 + eyz2));
  gz = 2.0 * axz + ((exz1 - exz2) + (eyz1 - eyz2));
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
template <bool WB, bool MOMENTS>
__global__ void __launch_bounds__(kBlock3) d3_collide(const double* __restrict__ src,
                                                      double* __restrict__ dst,
                                                      const double* __restrict__ rho,
                                                      const double* __restrict__ mu,
                                                      const P3 p, const Out3 out) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  const bool own = x < p.nx;
  double st[kStatRec] = {0.0, 0.0, 0.0, 1e300, -1e300, 0.0};
  if (own) {
    double g[kQ3];
#pragma unroll
    for (int i = 0; i < kQ3; ++i)
      g[i] = src[i * p.plane + at3(p, wrap3(x - cx3(i), p.nx), wrap3(y - cy3(i), p.ny),
                                   wrap3(z - cz3(i), p.nz))];
    const long long k = at3(p, x, y, z);
    const double r = rho[k];
    // 12 grad mu, 12 grad rho; F = -rho grad mu (Eq. mF), or the potential
    // form cs^2 grad rho - rho grad mu of the standard scheme
    double gmx, gmy, gmz, grx, gry, grz;
    grad3x12(mu, p, x, y, z, gmx, gmy, gmz);
    grad3x12(rho, p, x, y, z, grx, gry, grz);
    const double nr = r * (-1.0 / 12.0);
    double Fx, Fy, Fz;
    if (WB) {
      Fx = nr * gmx;
      Fy = nr * gmy;
      Fz = nr * gmz;
    } else {
      Fx = (1.0 / 36.0) * grx + nr * gmx;
      Fy = (1.0 / 36.0) * gry + nr * gmy;
      Fz = (1.0 / 36.0) * grz + nr * gmz;
    }
    // momentum from the differences of opposite pairs (each edge difference
    // serves two components)
    const double d12 = g[1] - g[2], d34 = g[3] - g[4], d56 = g[5] - g[6];
    const double d78 = g[7] - g[8], d910 = g[9] - g[10], d1112 = g[11] - g[12];
    const double d1314 = g[13] - g[14], d1516 = g[15] - g[16], d1718 = g[17] - g[18];
    const double jx = ((d12 + d78) + (d910 + d1112)) + d1314;
    const double jy = ((d34 + d78) - (d910 - d1516)) + d1718;
    const double jz = ((d56 + d1112) - (d1314 - d1516)) - d1718;
    const double inv = recip(r);
    const double ux = (jx + 0.5 * Fx) * inv, uy = (jy + 0.5 * Fy) * inv,
                 uz = (jz + 0.5 * Fz) * inv;                     // Eq. rhoU
    const double muc = mu[k];
    if (MOMENTS) {
      if (out.rho) out.rho[(size_t)(z * p.ny + y) * p.nx + x] = r;
      if (out.ux) out.ux[(size_t)(z * p.ny + y) * p.nx + x] = ux;
      if (out.uy) out.uy[(size_t)(z * p.ny + y) * p.nx + x] = uy;
      if (out.uz) out.uz[(size_t)(z * p.ny + y) * p.nx + x] = uz;
      if (out.mu) out.mu[(size_t)(z * p.ny + y) * p.nx + x] = muc;
      const double u2 = ux * ux + uy * uy + uz * uz;
      st[0] = r;
      st[1] = 0.5 * r * u2;
      st[2] = u2;
      st[3] = muc;
      st[4] = muc;
      st[5] = (!isfinite(r) || !isfinite(muc) || !isfinite(u2)) ? 1.0 : 0.0;
    } else {
      const double om = p.omega, kf = p.kforce;
      const double keep = 1.0 - om;
      double Gx = Fx, Gy = Fy, Gz = Fz;
      if (WB) {
        Gx = Fx + (1.0 / 36.0) * grx;                           // G = F + cs^2 grad rho
        Gy = Fy + (1.0 / 36.0) * gry;
        Gz = Fz + (1.0 / 36.0) * grz;
      }
      const double orho = om * r;
      const double t = -1.5 * orho * (ux * ux + uy * uy + uz * uz) -
                       3.0 * kf * (ux * Gx + uy * Gy + uz * Gz);
      const double ku = WB ? (kf * (1.0 / 12.0)) * (ux * grx + uy * gry + uz * grz) : 0.0;
      // per-node constants of the pairs, with the weights folded in
      // (w_ax = 1/18, w_edge = 1/36): E = C + cu (A cu + K.c), O = 3 w c.M
      const double Ca = WB ? (1.0 / 18.0) * t : (1.0 / 18.0) * (t + orho);
      const double Ce = WB ? (1.0 / 36.0) * (t + 1.5 * ku) : (1.0 / 36.0) * (t + orho);
      const double Aa = 0.25 * orho, Ae = 0.125 * orho;          // w 9/2 omega rho
      const double kh = 0.5 * kf, kq = 0.25 * kf, k6 = kf * (1.0 / 6.0);
      const double Kax = kh * Gx, Kay = kh * Gy, Kaz = kh * Gz;  // 9 w_ax kforce G
      const double Kex = kq * Gx, Key = kq * Gy, Kez = kq * Gz;  // 9 w_edge kforce G
      const double o6 = orho * (1.0 / 6.0);                      // 3 w_ax (omega rho u + kforce F)
      const double Mx = o6 * ux + k6 * Fx, My = o6 * uy + k6 * Fy, Mz = o6 * uz + k6 * Fz;
      auto axis = [&](int i, int j, double cu, double K, double M) {
        const double E = Ca + cu * (Aa * cu + K);
        g[i] = keep * g[i] + (E + M);
        g[j] = keep * g[j] + (E - M);
      };
      // edge pair: 3 w_edge c.M = (Ma + Mb) / 2 for c = a + b
      auto edge = [&](int i, int j, double cu, double K, double S) {
        const double E = Ce + cu * (Ae * cu + K);
        g[i] = keep * g[i] + (E + 0.5 * S);
        g[j] = keep * g[j] + (E - 0.5 * S);
      };
      axis(1, 2, ux, Kax, Mx);
      axis(3, 4, uy, Kay, My);
      axis(5, 6, uz, Kaz, Mz);
      edge(7, 8, ux + uy, Kex + Key, Mx + My);
      edge(9, 10, ux - uy, Kex - Key, Mx - My);
      edge(11, 12, ux + uz, Kex + Kez, Mx + Mz);
      edge(13, 14, ux - uz, Kex - Kez, Mx - Mz);
      edge(15, 16, uy + uz, Key + Kez, My + Mz);
      edge(17, 18, uy - uz, Key - Kez, My - Mz);
      // rest: WB f_0^eq - s_0 = rho - w_0 3/2 rho u.u, F_0 = w_0 (-3 u.G - 3/2 u.grad rho);
      // standard f_0^eq = w_0 rho (1 - 3/2 u.u), F_0 = w_0 (-3 u.G)
      const double w0 = 1.0 / 3.0;
      g[0] = keep * g[0] + (WB ? orho + w0 * (t - 1.5 * ku) : w0 * (t + orho));
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
__global__ void d3_init(const double* __restrict__ rho_in, double* __restrict__ dst, const P3 p,
                        int wb) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
#pragma unroll
  for (int i = 0; i < kQ3; ++i) {
    const int xx = wrap3(x + cx3(i), p.nx), yy = wrap3(y + cy3(i), p.ny),
              zz = wrap3(z + cz3(i), p.nz);
    const double r = rho_in[(size_t)(zz * p.ny + yy) * p.nx + xx];
    // WB: f_0^eq - s_0 = rho, f_i^eq - s_i = 0; standard: w_i rho
    dst[i * p.plane + at3(p, x, y, z)] = wb ? (i == 0 ? r : 0.0) : w3(i) * r;
  }
}

// f_i(x) = P_i(x - c_i) + s_i for one direction, [nz][ny][nx].
__global__ void d3_get(const double* __restrict__ src, double* __restrict__ f, const P3 p,
                       int dir, double shift) {
  const int x = blockIdx.x * kBlock3 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  const double v = src[dir * p.plane + at3(p, wrap3(x - cx3(dir), p.nx),
                                           wrap3(y - cy3(dir), p.ny), wrap3(z - cz3(dir), p.nz))];
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

Layout3 layout3(const wblbe3_params* p) {
  Layout3 L{};
  L.pitch = (p->nx + 15) / 16 * 16;
  L.plane = (long long)L.pitch * p->ny * p->nz;
  const size_t pops = align3((size_t)kQ3 * L.plane * sizeof(double));
  const size_t field = align3((size_t)L.plane * sizeof(double));
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
  double* buf[2];
  int cur;
  double *rho, *mu, *stage, *partials, *stats;
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
  return q;
}

dim3 grid3(const wblbe3_ctx* h) {
  return dim3((h->p.nx + kBlock3 - 1) / kBlock3, h->p.ny, h->p.nz);
}

double shift3(const wblbe3_params& p, int i) {
  if (p.scheme != WBLBE_WELL_BALANCED) return 0.0;
  return i == 0 ? -(1.0 - w3(0)) * p.rho0 : w3(i) * p.rho0;
}

// density and chemical potential of the current state, then the collision
// (step: into the other buffer) or the moments (fields and stats).
wblbe_status pass3(wblbe3_ctx* h, bool moments, const Out3& out) {
  const P3 q = p3_of(h);
  const dim3 g = grid3(h);
  d3_density<<<g, kBlock3, 0, h->stream>>>(h->buf[h->cur], h->rho, q);
  d3_chem_pot<<<g, kBlock3, 0, h->stream>>>(h->rho, h->mu, q);
  const bool wb = h->p.scheme == WBLBE_WELL_BALANCED;
  const double* src = h->buf[h->cur];
  double* dst = h->buf[1 - h->cur];
  if (moments) {
    if (wb) d3_collide<true, true><<<g, kBlock3, 0, h->stream>>>(src, nullptr, h->rho, h->mu, q, out);
    else d3_collide<false, true><<<g, kBlock3, 0, h->stream>>>(src, nullptr, h->rho, h->mu, q, out);
  } else {
    if (wb) d3_collide<true, false><<<g, kBlock3, 0, h->stream>>>(src, dst, h->rho, h->mu, q, out);
    else d3_collide<false, false><<<g, kBlock3, 0, h->stream>>>(src, dst, h->rho, h->mu, q, out);
  }
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
  h->buf[0] = reinterpret_cast<double*>(ws + L.off_a);
  h->buf[1] = reinterpret_cast<double*>(ws + L.off_b);
  h->rho = reinterpret_cast<double*>(ws + L.off_rho);
  h->mu = reinterpret_cast<double*>(ws + L.off_mu);
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
  d3_init<<<grid3(h), kBlock3, 0, h->stream>>>(src, h->buf[0], p3_of(h),
                                               h->p.scheme == WBLBE_WELL_BALANCED);
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
    d3_get<<<grid3(h), kBlock3, 0, h->stream>>>(h->buf[h->cur], dst, p3_of(h), i,
                                                shift3(h->p, i));
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
