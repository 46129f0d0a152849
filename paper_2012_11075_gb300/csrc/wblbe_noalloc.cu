// Allocation-free moments/statistics entry point (wblbe_moments_noalloc).
//
// Some callers cannot allocate device memory at all: hosts that pre-reserve
// the whole device for another allocator and forbid cudaMalloc, or plug-ins
// and callbacks that only ever see buffers handed to them.  For them this
// file keeps the only scratch the statistics reduction needs (one record per
// CTA plus the final record) in a file-scope __device__ array of fixed size.  Every GPU that loads the
// library holds that array until the process exits.
//
// The caller passes the populations f_i(x, t) (float64, [9][ny][nx], the
// layout of wblbe_get_populations) and receives rho, u, mu and the stats, as
// wblbe_moments would give for the same state.  The paper has no
// counterpart of this entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/wblbe.h"
#include "lbm_kernels.cuh"

using namespace wblbe;

namespace {

constexpr int kTileX = 32;                 // columns per CTA
constexpr int kTileY = 8;                  // rows per CTA
constexpr int kMaxRecords = 16384;         // CTA records the scratch holds
constexpr int kMaxDevices = 64;

// Scratch: kMaxRecords per-CTA records + one final record (6 doubles each).
__device__ __align__(256) double g_noalloc_scratch[(kMaxRecords + 1) * kStatRec];

// Host-side device addresses of g_noalloc_scratch, one per device, filled on
// the first call made with that device current.
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

thread_local char g_noalloc_error[256] = "";

wblbe_status noalloc_fail(wblbe_status st, const char* msg) {
  snprintf(g_noalloc_error, sizeof(g_noalloc_error), "%s", msg);
  return st;
}

// rho, mu, u and the stats of caller-layout populations (no streaming
// offsets: f_i(x) is read at x).  One CTA covers a kTileX x kTileY tile; the
// densities of the tile and a 2-node halo, then mu on a 1-node halo, are
// built in shared memory; the per-node velocity comes from the same
// collide() the step kernel uses (its post-collision output is discarded).
template <bool WB>
__global__ void __launch_bounds__(kTileX* kTileY)
    moments_noalloc_kernel(const double* __restrict__ f, KParams p, double* rho_out,
                           double* ux_out, double* uy_out, double* mu_out,
                           double* __restrict__ scratch) {
  __shared__ double rho_s[kTileY + 4][kTileX + 4];
  __shared__ double mu_s[kTileY + 2][kTileX + 2];
  __shared__ double red[kTileX * kTileY / 32][kStatRec];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int t = ty * kTileX + tx;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const long long plane = (long long)p.nx * p.ny;

  for (int q = t; q < (kTileY + 4) * (kTileX + 4); q += kTileX * kTileY) {
    const int ly = q / (kTileX + 4), lx = q % (kTileX + 4);
    const int gx = wrap_index(x0 - 2 + lx, p.nx), gy = wrap_index(y0 - 2 + ly, p.ny);
    const long long k = (long long)gy * p.nx + gx;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) s += f[i * plane + k];
    rho_s[ly][lx] = s;
  }
  __syncthreads();
  const double two_beta = p.two_beta, dl = p.dl, dg = p.dg, kappa6 = p.kappa / 6.0;
  for (int q = t; q < (kTileY + 2) * (kTileX + 2); q += kTileX * kTileY) {
    const int ly = q / (kTileX + 2) + 1, lx = q % (kTileX + 2) + 1;
    mu_s[ly - 1][lx - 1] = chem_pot<double>(
        rho_s[ly][lx], rho_s[ly][lx + 1], rho_s[ly][lx - 1], rho_s[ly + 1][lx],
        rho_s[ly - 1][lx], rho_s[ly + 1][lx + 1], rho_s[ly + 1][lx - 1],
        rho_s[ly - 1][lx + 1], rho_s[ly - 1][lx - 1], two_beta, dl, dg, kappa6);
  }
  __syncthreads();

  double v[kStatRec] = {0.0, 0.0, 0.0, 1e300, -1e300, 0.0};
  const int x = x0 + tx, y = y0 + ty;
  if (x < p.nx && y < p.ny) {
    const int ry = ty + 2, rx = tx + 2, my = ty + 1, mx = tx + 1;
    const double gmx = (1.0 / 3.0) * (mu_s[my][mx + 1] - mu_s[my][mx - 1]) +
                       (1.0 / 12.0) * ((mu_s[my + 1][mx + 1] + mu_s[my - 1][mx + 1]) -
                                       (mu_s[my + 1][mx - 1] + mu_s[my - 1][mx - 1]));
    const double gmy = (1.0 / 3.0) * (mu_s[my + 1][mx] - mu_s[my - 1][mx]) +
                       (1.0 / 12.0) * ((mu_s[my + 1][mx + 1] + mu_s[my + 1][mx - 1]) -
                                       (mu_s[my - 1][mx + 1] + mu_s[my - 1][mx - 1]));
    const double grx = (1.0 / 3.0) * (rho_s[ry][rx + 1] - rho_s[ry][rx - 1]) +
                       (1.0 / 12.0) * ((rho_s[ry + 1][rx + 1] + rho_s[ry - 1][rx + 1]) -
                                       (rho_s[ry + 1][rx - 1] + rho_s[ry - 1][rx - 1]));
    const double gry = (1.0 / 3.0) * (rho_s[ry + 1][rx] - rho_s[ry - 1][rx]) +
                       (1.0 / 12.0) * ((rho_s[ry + 1][rx + 1] + rho_s[ry + 1][rx - 1]) -
                                       (rho_s[ry - 1][rx + 1] + rho_s[ry - 1][rx - 1]));
    const long long k = (long long)y * p.nx + x;
    double g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = f[i * plane + k];
    const double rs = rho_s[ry][rx];
    double ux, uy;
    const CollideConsts<double> cc(p);
    collide<double, WB ? kSchWB : kSchStandard>(g, rs, gmx, gmy, grx, gry, cc, ux, uy);
    const double mu = mu_s[my][mx];
    if (rho_out) rho_out[k] = rs;
    if (ux_out) ux_out[k] = ux;
    if (uy_out) uy_out[k] = uy;
    if (mu_out) mu_out[k] = mu;
    const double u2 = ux * ux + uy * uy;
    v[0] = rs;
    v[1] = 0.5 * rs * u2;
    v[2] = u2;
    v[3] = mu;
    v[4] = mu;
    v[5] = (!isfinite(rs) || !isfinite(mu) || !isfinite(u2)) ? 1.0 : 0.0;
  }
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
  if ((t & 31) == 0)
#pragma unroll
    for (int q = 0; q < kStatRec; ++q) red[t >> 5][q] = v[q];
  __syncthreads();
  if (t == 0) {
    double r[kStatRec];
#pragma unroll
    for (int q = 0; q < kStatRec; ++q) r[q] = red[0][q];
    for (int w = 1; w < kTileX * kTileY / 32; ++w) {
      r[0] += red[w][0];
      r[1] += red[w][1];
      r[2] = fmax(r[2], red[w][2]);
      r[3] = fmin(r[3], red[w][3]);
      r[4] = fmax(r[4], red[w][4]);
      r[5] = fmax(r[5], red[w][5]);
    }
    double* out = scratch + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kStatRec;
#pragma unroll
    for (int q = 0; q < kStatRec; ++q) out[q] = r[q];
  }
}

// Set-up, once per device, with that device current: the device address of
// the scratch array (host code must not use the symbol itself).
wblbe_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(WBLBE_ECUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      snprintf(g_noalloc_error, sizeof(g_noalloc_error), "cudaGetSymbolAddress: %s",
               cudaGetErrorString(e));
      return WBLBE_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return WBLBE_OK;
}

}  // namespace

extern "C" {

wblbe_status wblbe_moments_noalloc(const wblbe_params* params, const double* f,
                                   double* rho, double* ux, double* uy, double* mu,
                                   wblbe_stats* stats, void* cuda_stream) {
  if (!params || !f) return noalloc_fail(WBLBE_EINVAL, "params and f must not be NULL");
  if (params->nx < 1 || params->ny < 1 || !(params->tau > 0.5) || !(params->beta > 0.0) ||
      !(params->kappa >= 0.0) || !(params->rho_g > 0.0) || !(params->rho_l > params->rho_g) ||
      (params->scheme != WBLBE_STANDARD && params->scheme != WBLBE_WELL_BALANCED))
    return noalloc_fail(WBLBE_EINVAL, "invalid parameters");
  if (params->precision != WBLBE_FP64)
    return noalloc_fail(WBLBE_EINVAL, "the allocation-free pass reads float64 populations: precision must be WBLBE_FP64");
  const long long gx = (params->nx + kTileX - 1) / kTileX;
  const long long gy = (params->ny + kTileY - 1) / kTileY;
  if (gx * gy > kMaxRecords || (long long)params->nx * params->ny >= (1LL << 31)) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "lattice %d x %d needs %lld scratch records; the fixed scratch holds %d "
             "(ceil(nx/32) * ceil(ny/8) <= %d)",
             params->nx, params->ny, gx * gy, kMaxRecords, kMaxRecords);
    return noalloc_fail(WBLBE_ENOMEM, msg);
  }
  double* scratch = nullptr;
  wblbe_status st = scratch_for_current_device(&scratch);
  if (st != WBLBE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  KParams kp{};
  kp.nx = params->nx;
  kp.ny = params->ny;
  kp.omega = 1.0 / params->tau;
  kp.kforce = 1.0 - 1.0 / (2.0 * params->tau);
  kp.kappa = params->kappa;
  kp.two_beta = 2.0 * params->beta;
  kp.dl = -params->rho_l;
  kp.dg = -params->rho_g;
  kp.rho_ref = 0.0;

  dim3 grid((unsigned)gx, (unsigned)gy), block(kTileX, kTileY);
  if (params->scheme == WBLBE_WELL_BALANCED)
    moments_noalloc_kernel<true><<<grid, block, 0, s>>>(f, kp, rho, ux, uy, mu, scratch);
  else
    moments_noalloc_kernel<false><<<grid, block, 0, s>>>(f, kp, rho, ux, uy, mu, scratch);
  cudaError_t e = cudaGetLastError();
  // every record the finalize reads was written above by this call, so the
  // previous call's contents need no clearing
  double* final_rec = scratch + (size_t)kMaxRecords * kStatRec;
  if (e == cudaSuccess) {
    stats_finalize_kernel<<<1, 256, 0, s>>>(scratch, (int)(gx * gy), final_rec);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(g_noalloc_error, sizeof(g_noalloc_error), "launch: %s", cudaGetErrorString(e));
    return WBLBE_ECUDA;
  }
  if (stats) {
    double v[kStatRec];
    e = cudaMemcpyAsync(v, final_rec, sizeof(v), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      snprintf(g_noalloc_error, sizeof(g_noalloc_error), "stats copy: %s", cudaGetErrorString(e));
      return WBLBE_ECUDA;
    }
    stats->step = 0;
    stats->mass = v[0];
    stats->kinetic = v[1];
    stats->umax = v[2];
    stats->mu_min = v[3];
    stats->mu_max = v[4];
    stats->nonfinite = v[5] != 0.0 || !std::isfinite(v[0]);
    stats->mass_drift_rel = 0.0;
  }
  return WBLBE_OK;
}

const char* wblbe_noalloc_last_error(void) { return g_noalloc_error; }

}  // extern "C"
