// The variants of the standard LBE that Sec. II of Guo, arXiv 2012.11075
// compares with: strip-kernel instantiations for the pressure-form
// interaction force (scheme code 2) and the forcing term of Guo's textbook
// (scheme code 3), and a tile kernel for the standard scheme with a
// sixth-order isotropic gradient in the force (scheme code 4, FP64).  The
// single-lattice runtime (wblbe.cu) dispatches to them.
#include "strip_launch.cuh"

namespace wblbe {

namespace {

// Scheme 4: standard LBE, potential-form force F = cs^2 grad(rho) - rho
// grad(mu) with both gradients taken by the radius-2 stencil on the shells
// |e|^2 = 1, 2, 4 whose weights 4/15, 1/10, 1/120 make the lattice moments
// isotropic to sixth order (normalisation sum W e_x^2 = 1 and the 4th- and
// 6th-order isotropy conditions).  A comparison scheme: one plain FP64 tile
// kernel, 32 x 16 nodes per CTA, densities over the tile plus 3 (pulled
// loads from device memory), mu over the tile plus 2, then the collision of
// the own nodes (the standard-scheme collision of the strip kernel).
constexpr int kE6Tx = 32, kE6Ty = 16, kE6Threads = 256;
constexpr int kRhoW = kE6Tx + 6, kRhoH = kE6Ty + 6;
constexpr int kMuW = kE6Tx + 4, kMuH = kE6Ty + 4;

__device__ __forceinline__ void grad_e6(const double* t, int w, int cx, int cy, double& gx,
                                        double& gy) {
  // t: tile with row width w; (cx, cy) the centre
  auto at = [&](int dx, int dy) { return t[(cy + dy) * w + cx + dx]; };
  const double w1 = 4.0 / 15.0, w2 = 1.0 / 10.0, w4 = 1.0 / 120.0;
  const double d1x = at(1, 0) - at(-1, 0), d1y = at(0, 1) - at(0, -1);
  const double a = at(1, 1), b = at(-1, 1), c = at(-1, -1), d = at(1, -1);
  const double d4x = at(2, 0) - at(-2, 0), d4y = at(0, 2) - at(0, -2);
  gx = w1 * d1x + w2 * ((a - b) + (d - c)) + 2.0 * w4 * d4x;
  gy = w1 * d1y + w2 * ((a + b) - (c + d)) + 2.0 * w4 * d4y;
}

__device__ __forceinline__ int e6_wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

template <int MODE>
__global__ void __launch_bounds__(kE6Threads)
    e6_tile_kernel(const double* __restrict__ src, double* __restrict__ dst, const KParams p,
                   const MomentsOut mo) {
  __shared__ double rho_t[kRhoH * kRhoW];
  __shared__ double mu_t[kMuH * kMuW];
  __shared__ double red[kE6Threads / 32][kStatRec];
  constexpr int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kE6Tx, y0 = blockIdx.y * kE6Ty;
  auto pulled = [&](int i, int x, int y) {
    return src[i * p.plane + (long long)e6_wrap(y - CY[i], p.ny) * p.pitch +
               e6_wrap(x - CX[i], p.nx)];
  };
  for (int k = tid; k < kRhoH * kRhoW; k += kE6Threads) {
    const int ly = k / kRhoW, lx = k - ly * kRhoW;
    const int x = e6_wrap(x0 - 3 + lx, p.nx), y = e6_wrap(y0 - 3 + ly, p.ny);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) s += pulled(i, x, y);
    rho_t[k] = s;
  }
  __syncthreads();
  const double two_beta = p.two_beta, dl = p.dl, dg = p.dg, kappa6 = p.kappa / 6.0;
  for (int k = tid; k < kMuH * kMuW; k += kE6Threads) {
    const int ly = k / kMuW, lx = k - ly * kMuW;
    const double* r = rho_t + (ly + 1) * kRhoW + lx + 1;
    mu_t[k] = chem_pot<double>(r[0], r[1], r[-1], r[kRhoW], r[-kRhoW], r[kRhoW + 1],
                               r[kRhoW - 1], r[-kRhoW + 1], r[-kRhoW - 1], two_beta, dl, dg,
                               kappa6);
  }
  __syncthreads();
  const CollideConsts<double> cc(p);
  StatsAcc acc;
  const bool acc_on = MODE != kModeStep;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int lx = tid & 31, ly = (tid >> 5) + 8 * half;
    const int x = x0 + lx, y = y0 + ly;
    if (x < p.nx && y < p.ny) {
      double gmx, gmy, grx, gry;
      grad_e6(mu_t, kMuW, lx + 2, ly + 2, gmx, gmy);
      grad_e6(rho_t, kRhoW, lx + 3, ly + 3, grx, gry);
      const double rs = rho_t[(ly + 3) * kRhoW + lx + 3];
      double g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = pulled(i, x, y);
      double ux, uy;
      collide<double, kSchStandard>(g, rs, gmx, gmy, grx, gry, cc, ux, uy);
      emit_node<double, MODE, false>(
          p, mo, dst, y, x, x, false, false, g, rs, mu_t[(ly + 2) * kMuW + lx + 2], ux, uy,
          acc, acc_on);
    }
  }
  if (MODE != kModeStep && mo.partials) {
    double v[kStatRec] = {acc.mass, acc.kin, acc.u2, acc.mumin, acc.mumax, (double)acc.bad};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o0 = __shfl_down_sync(0xffffffffu, v[0], off);
      const double o1 = __shfl_down_sync(0xffffffffu, v[1], off);
      const double o2 = __shfl_down_sync(0xffffffffu, v[2], off);
      const double o3 = __shfl_down_sync(0xffffffffu, v[3], off);
      const double o4 = __shfl_down_sync(0xffffffffu, v[4], off);
      const double o5 = __shfl_down_sync(0xffffffffu, v[5], off);
      v[0] += o0;
      v[1] += o1;
      v[2] = fmax(v[2], o2);
      v[3] = fmin(v[3], o3);
      v[4] = fmax(v[4], o4);
      v[5] = fmax(v[5], o5);
    }
    if ((tid & 31) == 0)
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) red[tid >> 5][q] = v[q];
    __syncthreads();
    if (tid == 0) {
      double r[kStatRec];
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) r[q] = red[0][q];
      for (int w = 1; w < kE6Threads / 32; ++w) {
        r[0] += red[w][0];
        r[1] += red[w][1];
        r[2] = fmax(r[2], red[w][2]);
        r[3] = fmin(r[3], red[w][3]);
        r[4] = fmax(r[4], red[w][4]);
        r[5] = fmax(r[5], red[w][5]);
      }
      double* out = mo.partials + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kStatRec;
#pragma unroll
      for (int q = 0; q < kStatRec; ++q) out[q] = r[q];
    }
  }
}

}  // namespace

int e6_partials(int nx, int ny) {
  return ((nx + kE6Tx - 1) / kE6Tx) * ((ny + kE6Ty - 1) / kE6Ty);
}

cudaError_t launch_e6(int mode, const void* src, void* dst, const KParams& kp,
                      const MomentsOut& mo, cudaStream_t s) {
  dim3 grid((kp.nx + kE6Tx - 1) / kE6Tx, (kp.ny + kE6Ty - 1) / kE6Ty);
  const double* in = static_cast<const double*>(src);
  double* out = static_cast<double*>(dst);
  switch (mode) {
    case kModeStep: e6_tile_kernel<kModeStep><<<grid, kE6Threads, 0, s>>>(in, out, kp, mo); break;
    case kModeMoments: e6_tile_kernel<kModeMoments><<<grid, kE6Threads, 0, s>>>(in, out, kp, mo); break;
    case kModeStepStats:
      e6_tile_kernel<kModeStepStats><<<grid, kE6Threads, 0, s>>>(in, out, kp, mo);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_variant(int sch, bool fp64, int mode, const void* src, void* dst,
                           const KParams& kp, const MomentsOut& mo, int tile, cudaStream_t s) {
  if (sch == kSchPressure)
    return launch_scheme<kSchPressure>(fp64, mode, src, dst, kp, mo, tile, s);
  if (sch == kSchTextbook)
    return launch_scheme<kSchTextbook>(fp64, mode, src, dst, kp, mo, tile, s);
  return cudaErrorInvalidValue;
}

int resident_variant(int sch, bool fp64, int tile) {
  return sch == kSchPressure ? resident_scheme<kSchPressure>(fp64, tile)
                             : resident_scheme<kSchTextbook>(fp64, tile);
}

unsigned int variants_bounds_errors(bool reset) { return read_bounds_errors(reset); }

cudaError_t allow_smem_variants() {
  cudaError_t e = cudaSuccess, r;
  if ((r = allow_smem_scheme<kSchPressure>()) != cudaSuccess) e = r;
  if ((r = allow_smem_scheme<kSchTextbook>()) != cudaSuccess) e = r;
  return e;
}

}  // namespace wblbe
