// C-ABI runtime of the well-balanced / standard D2Q9 LBE library
// (declarations and conventions in include/wblbe.h).
//
// A handle owns no device memory: it carves the caller's workspace into two
// population buffers (ping-pong), one float64 staging field for host I/O,
// per-CTA reduction partials and a stats record.  Steps are issued on the
// caller's stream; chunks of steps are captured once into a CUDA graph and
// replayed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/wblbe.h"
#include "lbm_kernels.cuh"
#include "strip_launch.cuh"

using namespace wblbe;

namespace {

constexpr size_t kAlign = 256;
constexpr int kGraphSteps = 32;          // steps per captured graph (even)
constexpr int kMomentsRows = 16;         // rows per CTA of the moments kernel
constexpr int kNumSMs = 152;

thread_local char g_thread_error[256] = "";

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  int pitch;            // elements per row
  size_t elem;          // bytes per population element
  long long plane;      // elements per plane
  size_t pops_bytes;    // one population buffer
  size_t off_a, off_b, off_stage, off_partials, off_stats, off_step, total;
  int max_partials;
};

bool params_valid(const wblbe_params* p, char* why, size_t n) {
  if (!p) { snprintf(why, n, "params is NULL"); return false; }
  if (p->nx < 1 || p->ny < 1) { snprintf(why, n, "nx, ny must be >= 1"); return false; }
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) { snprintf(why, n, "tau must be > 0.5"); return false; }
  if (!(p->kappa >= 0.0) || !std::isfinite(p->kappa)) { snprintf(why, n, "kappa must be >= 0"); return false; }
  if (!(p->beta > 0.0) || !std::isfinite(p->beta)) { snprintf(why, n, "beta must be > 0"); return false; }
  if (!(p->rho_g > 0.0) || !(p->rho_l > p->rho_g) || !std::isfinite(p->rho_l)) {
    snprintf(why, n, "need rho_l > rho_g > 0"); return false;
  }
  if (!std::isfinite(p->rho0)) { snprintf(why, n, "rho0 must be finite"); return false; }
  if (p->scheme < WBLBE_STANDARD || p->scheme > WBLBE_STANDARD_E6) {
    snprintf(why, n, "unknown scheme %d", p->scheme); return false;
  }
  if (p->scheme == WBLBE_STANDARD_E6 && p->precision != WBLBE_FP64) {
    snprintf(why, n, "the E6 comparison scheme runs in FP64 only"); return false;
  }
  if (p->precision != WBLBE_FP64 && p->precision != WBLBE_FP32_SHIFTED) {
    snprintf(why, n, "unknown precision %d", p->precision); return false;
  }
  if (p->precision == WBLBE_FP32_SHIFTED && std::isinf(p->rho_ref)) {
    snprintf(why, n, "rho_ref must be finite or NaN"); return false;
  }
  return true;
}

Layout make_layout(const wblbe_params* p) {
  Layout L{};
  L.elem = p->precision == WBLBE_FP64 ? 8 : 4;
  const int align_elems = (int)(128 / L.elem);
  L.pitch = (p->nx + align_elems - 1) / align_elems * align_elems;
  L.plane = (long long)L.pitch * p->ny;
  L.pops_bytes = align_up((size_t)9 * (size_t)L.plane * L.elem);
  // per-CTA records: the moments pass (32-column strips at the narrowest,
  // kMomentsRows rows) and a step with statistics in any default launch
  // shape (at least 32 columns and 8 rows per CTA)
  const int strips = (p->nx + 31) / 32;
  const int runs = (p->ny + 7) / 8;
  L.max_partials = strips * runs;
  size_t off = 0;
  L.off_a = off; off += L.pops_bytes;
  L.off_b = off; off += L.pops_bytes;
  L.off_stage = off; off += align_up((size_t)p->nx * p->ny * sizeof(double));
  L.off_partials = off; off += align_up((size_t)L.max_partials * kStatRec * sizeof(double));
  L.off_stats = off; off += align_up(8 * sizeof(double));
  L.off_step = off; off += align_up(sizeof(long long));
  L.total = off;
  return L;
}

}  // namespace

struct wblbe_ctx {
  wblbe_params p;
  Layout L;
  int device;
  cudaStream_t stream;
  cudaStream_t capture_stream;
  unsigned char* ws;
  void* buf[2];
  int cur;                       // buffer holding the state
  double* stage;
  double* partials;
  double* stats_dev;
  long long* step_dev;           // step of the first step of a graph replay
  wblbe_launch launch;
  int64_t steps;
  int64_t launches;
  double mass0;
  bool have_state;
  cudaGraphExec_t graph;         // kGraphSteps steps starting from buf[0]
  bool graph_valid;
  char err[256];
};

namespace {

wblbe_status fail(wblbe_ctx* h, wblbe_status st, const char* fmt, ...) {
  char* dst = h ? h->err : g_thread_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 256, fmt, ap);
  va_end(ap);
  return st;
}

#define CU(h, call)                                                          \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return fail((h), WBLBE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Keeps the caller's current device and switches to the handle's.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// FP32 shift density; by default the gas density: the rest population is
// stored as g_0 ~ rho - rho_ref, so the low-density phase, where an absolute
// rounding of g_0 weighs most, gets the finest resolution (measured against
// FP64 on the 4096^2 droplet case after 10000 steps: velocity error 17-27x
// and mass drift up to 20x smaller than with the mean density).
double rho_ref_of(const wblbe_params& p) {
  if (p.precision == WBLBE_FP64) return 0.0;
  return std::isnan(p.rho_ref) ? p.rho_g : p.rho_ref;
}

KParams make_kparams(const wblbe_ctx* h, int rows) {
  const wblbe_params& p = h->p;
  KParams k{};
  k.nx = p.nx;
  k.ny = p.ny;
  k.pitch = h->L.pitch;
  k.rows = rows;
  k.plane = h->L.plane;
  k.omega = 1.0 / p.tau;
  k.kforce = 1.0 - 1.0 / (2.0 * p.tau);
  k.kappa = p.kappa;
  k.two_beta = 2.0 * p.beta;
  const double rr = rho_ref_of(p);
  k.rho_ref = rr;
  k.dl = rr - p.rho_l;
  k.dg = rr - p.rho_g;
  k.row_lo = 0;
  k.row_hi = p.ny;
  k.y_offset = 0;
  return k;
}

// The stored shift s_i of a parameter set (see make_layout_params).
void shift_of(const wblbe_params& p, double s[9]) {
  const double w[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
  const double rr = rho_ref_of(p);
  for (int i = 0; i < 9; ++i) {
    if (p.scheme == WBLBE_WELL_BALANCED)
      s[i] = (i == 0) ? rr - (1.0 - w[0]) * p.rho0 : w[i] * p.rho0;
    else
      s[i] = w[i] * rr;
  }
}

LayoutParams make_layout_params(const wblbe_ctx* h) {
  const wblbe_params& p = h->p;
  LayoutParams lp{};
  lp.nx = p.nx;
  lp.ny = p.ny;
  lp.pitch = h->L.pitch;
  lp.plane = h->L.plane;
  lp.wb = p.scheme == WBLBE_WELL_BALANCED;
  lp.rho0 = p.rho0;
  // the rest equilibrium at rho_ref (0 in FP64); it carries the WB rho0
  // vector in both precisions, so the kernel never sees rho0
  shift_of(p, lp.shift);
  return lp;
}

bool launch_valid(const wblbe_launch* l) {
  if (!l) return false;
  if (l->tile_x != 32 && l->tile_x != 64 && l->tile_x != 128 && l->tile_x != 256) return false;
  return l->rows_per_cta >= 1;
}

// Scheme codes 0 (standard) and 1 (well-balanced) are instantiated here, the
// comparison variants 2 and 3 in strip_variants.cu.
cudaError_t allow_smem_all() {
  cudaError_t e = cudaSuccess, r;
  if ((r = allow_smem_scheme<kSchStandard>()) != cudaSuccess) e = r;
  if ((r = allow_smem_scheme<kSchWB>()) != cudaSuccess) e = r;
  if ((r = allow_smem_variants()) != cudaSuccess) e = r;
  return e;
}

int resident_for(const wblbe_params& p, int tile) {
  const bool fp64 = p.precision == WBLBE_FP64;
  switch (p.scheme) {
    case WBLBE_STANDARD: return resident_scheme<kSchStandard>(fp64, tile);
    case WBLBE_WELL_BALANCED: return resident_scheme<kSchWB>(fp64, tile);
    case WBLBE_STANDARD_E6: return 1;      // fixed tiles; the launch shape is not used
    default: return resident_variant(p.scheme, fp64, tile);
  }
}

// Default launch shape: 128-column strips (narrower lattices: 64 or 32), and
// rows per CTA chosen so that the whole grid is resident at once (one wave),
// with at least 8 rows per CTA (each CTA re-reads 4 halo rows).
wblbe_launch default_launch(const wblbe_params& p) {
  wblbe_launch l{};
  l.tile_x = p.nx >= 128 ? 128 : (p.nx > 32 ? 64 : 32);
  int nsm = kNumSMs, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = resident_for(p, l.tile_x);
  const long long resident = (long long)per_sm * nsm;
  const long long strips = (p.nx + l.tile_x - 1) / l.tile_x;
  long long segs = resident / strips;
  if (segs < 1) segs = 1;
  long long rows = (p.ny + segs - 1) / segs;
  if (rows < 8) rows = 8;
  rows += rows & 1;          // even: every CTA starts on an even row (see pair_uniforms)
  if (rows > p.ny) rows = p.ny;
  l.rows_per_cta = (int)rows;
  return l;
}

// mode: kModeStep, kModeMoments or kModeStepStats (see StripMode)
cudaError_t launch_any(const wblbe_ctx* h, int mode, const void* src,
                       void* dst, const KParams& kp, const MomentsOut& mo,
                       int tile, cudaStream_t s) {
  const bool fp64 = h->p.precision == WBLBE_FP64;
  switch (h->p.scheme) {
    case WBLBE_STANDARD:
      return launch_scheme<kSchStandard>(fp64, mode, src, dst, kp, mo, tile, s);
    case WBLBE_WELL_BALANCED:
      return launch_scheme<kSchWB>(fp64, mode, src, dst, kp, mo, tile, s);
    case WBLBE_STANDARD_E6:
      return launch_e6(mode, src, dst, kp, mo, s);
    default:
      return launch_variant(h->p.scheme, fp64, mode, src, dst, kp, mo, tile, s);
  }
}

// Per-CTA statistics records a step launch writes in the step-with-statistics
// mode (the E6 tile kernel uses fixed 32 x 16 tiles).
long long step_records(const wblbe_ctx* h) {
  if (h->p.scheme == WBLBE_STANDARD_E6) return e6_partials(h->p.nx, h->p.ny);
  const long long tx = h->launch.tile_x, rows = h->launch.rows_per_cta;
  return ((h->p.nx + tx - 1) / tx) * ((h->p.ny + rows - 1) / rows);
}

// One step from buf[from] to buf[1-from] on stream s.  The time step of the
// state it updates: h->steps for a direct launch; for step k of a captured
// graph, k plus the base that the replay finds in h->step_dev.
cudaError_t issue_step(wblbe_ctx* h, int from, cudaStream_t s, int graph_k = -1) {
  KParams kp = make_kparams(h, h->launch.rows_per_cta);
  if (graph_k >= 0) {
    kp.step = graph_k;
    kp.step_base = h->step_dev;
  } else {
    kp.step = h->steps;
  }
  MomentsOut mo{};
  return launch_any(h, kModeStep, h->buf[from], h->buf[1 - from], kp, mo,
                    h->launch.tile_x, s);
}

__global__ void set_step_kernel(long long* dst, long long v) { *dst = v; }

void drop_graph(wblbe_ctx* h) {
  if (h->graph_valid) cudaGraphExecDestroy(h->graph);
  h->graph_valid = false;
}

wblbe_status build_graph(wblbe_ctx* h) {
  drop_graph(h);
  cudaGraph_t g = nullptr;
  CU(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k)
    le = issue_step(h, k & 1, h->capture_stream, k);
  cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(h, WBLBE_ECUDA, "graph capture failed: %s",
                cudaGetErrorString(le != cudaSuccess ? le : ce));
  }
  cudaError_t ie = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess)
    return fail(h, WBLBE_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
  h->graph_valid = true;
  return WBLBE_OK;
}

// Moments pass over the current state into device fields (any may be null)
// and its statistics record (stats_out, or the handle's record).
wblbe_status run_moments(wblbe_ctx* h, double* rho, double* ux, double* uy,
                         double* mu, double* stats_out = nullptr) {
  const int tile = h->p.nx >= 128 ? 128 : (h->p.nx > 32 ? 64 : 32);
  KParams kp = make_kparams(h, kMomentsRows);
  MomentsOut mo{rho, ux, uy, mu, h->partials};
  CU(h, launch_any(h, kModeMoments, h->buf[h->cur], nullptr, kp, mo, tile, h->stream));
  const int n = h->p.scheme == WBLBE_STANDARD_E6
                    ? e6_partials(h->p.nx, h->p.ny)
                    : ((h->p.nx + tile - 1) / tile) * ((h->p.ny + kMomentsRows - 1) / kMomentsRows);
  stats_finalize_kernel<<<1, 256, 0, h->stream>>>(h->partials, n,
                                                  stats_out ? stats_out : h->stats_dev);
  CU(h, cudaGetLastError());
  h->launches += 2;
  return WBLBE_OK;
}

wblbe_status read_stats(wblbe_ctx* h, wblbe_stats* out) {
  double v[kStatRec];
  CU(h, cudaMemcpyAsync(v, h->stats_dev, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (out) {
    out->step = h->steps;
    out->mass = v[0];
    out->kinetic = v[1];
    out->umax = v[2];
    out->mu_min = v[3];
    out->mu_max = v[4];
    out->nonfinite = v[5] != 0.0 || !std::isfinite(v[0]);
    out->mass_drift_rel = h->mass0 != 0.0 ? (v[0] - h->mass0) / h->mass0 : 0.0;
  }
  return WBLBE_OK;
}

// One step from the current state in the step-with-statistics mode: the
// kernel reduces the statistics of the state f(t) it starts from (the same
// rho, u and mu a moments pass computes) while it writes f(t+1) to the other
// buffer.  The handle keeps f(t) until the caller adopts the step with
// adopt_stats_step; the statistics land in h->stats_dev.  Needs
// step_records(h) <= the workspace's record capacity.
wblbe_status stats_step(wblbe_ctx* h) {
  KParams kp = make_kparams(h, h->launch.rows_per_cta);
  kp.step = h->steps;
  MomentsOut mo{};
  mo.partials = h->partials;
  CU(h, launch_any(h, kModeStepStats, h->buf[h->cur], h->buf[1 - h->cur], kp, mo,
                   h->launch.tile_x, h->stream));
  stats_finalize_kernel<<<1, 256, 0, h->stream>>>(h->partials, (int)step_records(h),
                                                  h->stats_dev);
  CU(h, cudaGetLastError());
  h->launches += 2;
  return WBLBE_OK;
}

void adopt_stats_step(wblbe_ctx* h) {
  h->cur ^= 1;
  h->steps += 1;
}

wblbe_status reset_mass(wblbe_ctx* h) {
  wblbe_status st = run_moments(h, nullptr, nullptr, nullptr, nullptr);
  if (st != WBLBE_OK) return st;
  wblbe_stats s{};
  st = read_stats(h, &s);
  if (st != WBLBE_OK) return st;
  h->mass0 = s.mass;
  return WBLBE_OK;
}

dim3 layout_grid(const wblbe_ctx* h) {
  return dim3((h->p.nx + 127) / 128, h->p.ny);
}

}  // namespace

namespace wblbe {

cudaError_t launch_strip_any(int sch, bool fp64, int mode, const void* src, void* dst,
                             const KParams& kp, const MomentsOut& mo, int tile, cudaStream_t s) {
  switch (sch) {
    case WBLBE_STANDARD: return launch_scheme<kSchStandard>(fp64, mode, src, dst, kp, mo, tile, s);
    case WBLBE_WELL_BALANCED: return launch_scheme<kSchWB>(fp64, mode, src, dst, kp, mo, tile, s);
    case WBLBE_STANDARD_PRESSURE:
    case WBLBE_STANDARD_TEXTBOOK:
      return launch_variant(sch, fp64, mode, src, dst, kp, mo, tile, s);
    default: return cudaErrorInvalidValue;
  }
}

int resident_strip_any(int sch, bool fp64, int tile) {
  switch (sch) {
    case WBLBE_STANDARD: return resident_scheme<kSchStandard>(fp64, tile);
    case WBLBE_WELL_BALANCED: return resident_scheme<kSchWB>(fp64, tile);
    default: return resident_variant(sch, fp64, tile);
  }
}

cudaError_t allow_smem_strip_all() { return allow_smem_all(); }

}  // namespace wblbe

extern "C" {

size_t wblbe_workspace_bytes(const wblbe_params* params) {
  char why[256];
  if (!params_valid(params, why, sizeof(why))) return 0;
  if ((long long)params->ny * ((params->nx + 31) / 32 * 32) >= (1LL << 31)) return 0;
  return make_layout(params).total;
}

wblbe_status wblbe_create(const wblbe_params* params, void* dev_workspace,
                          size_t workspace_bytes, void* cuda_stream,
                          wblbe_handle* out) {
  char why[256];
  if (!out) return fail(nullptr, WBLBE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params_valid(params, why, sizeof(why))) return fail(nullptr, WBLBE_EINVAL, "%s", why);
  const size_t need = wblbe_workspace_bytes(params);
  if (need == 0) return fail(nullptr, WBLBE_EINVAL, "lattice too large");
  if (!dev_workspace || ((uintptr_t)dev_workspace % kAlign) != 0)
    return fail(nullptr, WBLBE_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < need)
    return fail(nullptr, WBLBE_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
  wblbe_ctx* h = new (std::nothrow) wblbe_ctx();
  if (!h) return fail(nullptr, WBLBE_ENOMEM, "host allocation failed");
  h->p = *params;
  h->L = make_layout(params);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return fail(nullptr, WBLBE_ECUDA, "no CUDA device");
  }
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  {
    cudaError_t e = allow_smem_all();
    if (e != cudaSuccess) {
      delete h;
      return fail(nullptr, WBLBE_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    }
  }
  if (cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return fail(nullptr, WBLBE_ECUDA, "cudaStreamCreate failed");
  }
  h->ws = static_cast<unsigned char*>(dev_workspace);
  h->buf[0] = h->ws + h->L.off_a;
  h->buf[1] = h->ws + h->L.off_b;
  h->stage = reinterpret_cast<double*>(h->ws + h->L.off_stage);
  h->partials = reinterpret_cast<double*>(h->ws + h->L.off_partials);
  h->stats_dev = reinterpret_cast<double*>(h->ws + h->L.off_stats);
  h->step_dev = reinterpret_cast<long long*>(h->ws + h->L.off_step);
  h->cur = 0;
  h->launch = default_launch(*params);
  *out = h;
  return WBLBE_OK;
}

wblbe_status wblbe_set_params(wblbe_handle h, const wblbe_params* params) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  char why[256];
  if (!params_valid(params, why, sizeof(why))) return fail(h, WBLBE_EINVAL, "%s", why);
  if (params->nx != h->p.nx || params->ny != h->p.ny || params->precision != h->p.precision)
    return fail(h, WBLBE_EINVAL, "nx, ny and precision are fixed for a handle");
  {
    // the stored state is a deviation from the shift: it may not change
    double s_old[9], s_new[9];
    shift_of(h->p, s_old);
    shift_of(*params, s_new);
    for (int i = 0; i < 9; ++i)
      if (s_old[i] != s_new[i])
        return fail(h, WBLBE_EINVAL,
                    "the storage shift (rho_ref and scheme in FP32, rho0 of the "
                    "well-balanced scheme) is fixed for a handle");
  }
  h->p = *params;
  drop_graph(h);
  return WBLBE_OK;
}

wblbe_status wblbe_set_launch(wblbe_handle h, const wblbe_launch* launch) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!launch_valid(launch)) return fail(h, WBLBE_EINVAL, "tile_x must be 32/64/128/256 and rows_per_cta >= 1");
  h->launch = *launch;
  drop_graph(h);
  return WBLBE_OK;
}

wblbe_status wblbe_get_launch(wblbe_handle h, wblbe_launch* launch) {
  if (!h || !launch) return fail(h, WBLBE_EINVAL, "NULL argument");
  *launch = h->launch;
  return WBLBE_OK;
}

}  // extern "C"

namespace {

// f = f^eq(rho, 0) from a device field, on the handle's stream.
wblbe_status issue_init(wblbe_ctx* h, const double* src) {
  LayoutParams lp = make_layout_params(h);
  h->cur = 0;
  if (h->p.precision == WBLBE_FP64)
    init_rest_kernel<double><<<layout_grid(h), 128, 0, h->stream>>>(src, (double*)h->buf[0], lp);
  else
    init_rest_kernel<float><<<layout_grid(h), 128, 0, h->stream>>>(src, (float*)h->buf[0], lp);
  CU(h, cudaGetLastError());
  h->launches += 1;
  h->steps = 0;
  h->have_state = true;
  return WBLBE_OK;
}

}  // namespace

extern "C" {

wblbe_status wblbe_init_rho(wblbe_handle h, const double* rho, int32_t rho_on_device) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!rho) return fail(h, WBLBE_EINVAL, "rho is NULL");
  DeviceGuard dg(h->device);
  const double* src = rho;
  if (!rho_on_device) {
    CU(h, cudaMemcpyAsync(h->stage, rho, (size_t)h->p.nx * h->p.ny * sizeof(double),
                          cudaMemcpyHostToDevice, h->stream));
    src = h->stage;
  }
  wblbe_status st = issue_init(h, src);
  if (st != WBLBE_OK) return st;
  return reset_mass(h);
}

wblbe_status wblbe_step(wblbe_handle h, int64_t nsteps) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, WBLBE_EINVAL, "nsteps must be >= 0");
  if (!h->have_state) return fail(h, WBLBE_EINVAL, "no state: call wblbe_init_rho first");
  DeviceGuard dg(h->device);
  int64_t left = nsteps;
  if (left >= kGraphSteps) {
    if (!h->graph_valid) {
      wblbe_status st = build_graph(h);
      if (st != WBLBE_OK) return st;
    }
    // The graph alternates buf[0] -> buf[1] -> ...; with the state in buf[1]
    // one direct step first brings it back to buf[0].
    if (h->cur == 1) {
      CU(h, issue_step(h, 1, h->stream));
      h->cur = 0;
      h->launches += 1;
      h->steps += 1;
      --left;
    }
    while (left >= kGraphSteps) {
      set_step_kernel<<<1, 1, 0, h->stream>>>(h->step_dev, h->steps);
      CU(h, cudaGetLastError());
      CU(h, cudaGraphLaunch(h->graph, h->stream));
      h->launches += kGraphSteps + 1;
      h->steps += kGraphSteps;
      left -= kGraphSteps;
    }
  }
  // the step count follows what was issued, also when a launch fails midway
  for (; left > 0; --left) {
    CU(h, issue_step(h, h->cur, h->stream));
    h->cur ^= 1;
    h->launches += 1;
    h->steps += 1;
  }
  return WBLBE_OK;
}

wblbe_status wblbe_moments(wblbe_handle h, double* rho, double* ux, double* uy,
                           double* mu, int32_t out_on_device, wblbe_stats* stats) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!h->have_state) return fail(h, WBLBE_EINVAL, "no state: call wblbe_init_rho first");
  DeviceGuard dg(h->device);
  wblbe_status st;
  if (out_on_device) {
    st = run_moments(h, rho, ux, uy, mu);
    if (st != WBLBE_OK) return st;
  } else {
    double* outs[4] = {rho, ux, uy, mu};
    bool any = false;
    const size_t bytes = (size_t)h->p.nx * h->p.ny * sizeof(double);
    for (int k = 0; k < 4; ++k) {
      if (!outs[k]) continue;
      any = true;
      double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
      dev[k] = h->stage;
      st = run_moments(h, dev[0], dev[1], dev[2], dev[3]);
      if (st != WBLBE_OK) return st;
      CU(h, cudaMemcpyAsync(outs[k], h->stage, bytes, cudaMemcpyDeviceToHost, h->stream));
    }
    if (!any) {
      st = run_moments(h, nullptr, nullptr, nullptr, nullptr);
      if (st != WBLBE_OK) return st;
    }
  }
  return read_stats(h, stats);
}

wblbe_status wblbe_run_until_equilibrium(wblbe_handle h, double umax_tol,
                                         int64_t max_steps, int64_t check_every,
                                         int64_t* steps_done, wblbe_stats* out) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (check_every < 1 || max_steps < 0 || !(umax_tol >= 0.0))
    return fail(h, WBLBE_EINVAL, "need check_every >= 1, max_steps >= 0, umax_tol >= 0");
  if (steps_done) *steps_done = 0;
  if (!h->have_state) return fail(h, WBLBE_EINVAL, "no state: call wblbe_init_rho first");
  DeviceGuard dg(h->device);
  // A check reduces the statistics inside the step that leaves the checked
  // state (no separate pass over the nine planes): that step writes f(t+1)
  // to the other buffer, and is adopted as the first step of the next chunk
  // unless the run stops at this check, in which case the state stays f(t).
  // Lattices whose step grid has more CTAs than the workspace has records
  // (launch shapes with very few rows per CTA) fall back to a moments pass.
  const bool fused = step_records(h) <= h->L.max_partials;
  int64_t done = 0;
  wblbe_stats s{};
  for (;;) {
    wblbe_status st = fused ? stats_step(h)
                            : run_moments(h, nullptr, nullptr, nullptr, nullptr);
    if (st != WBLBE_OK) return st;
    st = read_stats(h, &s);
    if (st != WBLBE_OK) return st;
    if (out) *out = s;
    if (steps_done) *steps_done = done;
    if (s.nonfinite) return fail(h, WBLBE_EUNSTABLE, "non-finite value at step %lld", (long long)s.step);
    if (s.umax < umax_tol) return WBLBE_OK;
    if (done >= max_steps) return fail(h, WBLBE_ENOTCONVERGED, "max|u| = %g after %lld steps", s.umax, (long long)done);
    int64_t n = check_every < max_steps - done ? check_every : max_steps - done;
    if (fused) {
      adopt_stats_step(h);
      done += 1;
      n -= 1;
    }
    st = wblbe_step(h, n);
    if (st != WBLBE_OK) return st;
    done += n;
  }
}

wblbe_status wblbe_get_populations(wblbe_handle h, double* f, int32_t on_device) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!f) return fail(h, WBLBE_EINVAL, "f is NULL");
  if (!h->have_state) return fail(h, WBLBE_EINVAL, "no state: call wblbe_init_rho first");
  DeviceGuard dg(h->device);
  LayoutParams lp = make_layout_params(h);
  const size_t field = (size_t)h->p.nx * h->p.ny;
  const bool fp64 = h->p.precision == WBLBE_FP64;
  if (on_device) {
    if (fp64) get_pops_kernel<double><<<layout_grid(h), 128, 0, h->stream>>>((const double*)h->buf[h->cur], f, lp, 0, 9);
    else get_pops_kernel<float><<<layout_grid(h), 128, 0, h->stream>>>((const float*)h->buf[h->cur], f, lp, 0, 9);
    CU(h, cudaGetLastError());
    h->launches += 1;
  } else {
    for (int i = 0; i < 9; ++i) {
      if (fp64) get_pops_kernel<double><<<layout_grid(h), 128, 0, h->stream>>>((const double*)h->buf[h->cur], h->stage, lp, i, 1);
      else get_pops_kernel<float><<<layout_grid(h), 128, 0, h->stream>>>((const float*)h->buf[h->cur], h->stage, lp, i, 1);
      CU(h, cudaGetLastError());
      h->launches += 1;
      CU(h, cudaMemcpyAsync(f + i * field, h->stage, field * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
  }
  CU(h, cudaStreamSynchronize(h->stream));
  return WBLBE_OK;
}

wblbe_status wblbe_set_populations(wblbe_handle h, const double* f, int32_t on_device) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!f) return fail(h, WBLBE_EINVAL, "f is NULL");
  DeviceGuard dg(h->device);
  LayoutParams lp = make_layout_params(h);
  const size_t field = (size_t)h->p.nx * h->p.ny;
  const bool fp64 = h->p.precision == WBLBE_FP64;
  h->cur = 0;
  if (on_device) {
    if (fp64) set_pops_kernel<double><<<layout_grid(h), 128, 0, h->stream>>>(f, (double*)h->buf[0], lp, 0, 9);
    else set_pops_kernel<float><<<layout_grid(h), 128, 0, h->stream>>>(f, (float*)h->buf[0], lp, 0, 9);
    CU(h, cudaGetLastError());
    h->launches += 1;
  } else {
    for (int i = 0; i < 9; ++i) {
      CU(h, cudaMemcpyAsync(h->stage, f + i * field, field * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      if (fp64) set_pops_kernel<double><<<layout_grid(h), 128, 0, h->stream>>>(h->stage, (double*)h->buf[0], lp, i, 1);
      else set_pops_kernel<float><<<layout_grid(h), 128, 0, h->stream>>>(h->stage, (float*)h->buf[0], lp, i, 1);
      CU(h, cudaGetLastError());
      h->launches += 1;
    }
  }
  h->have_state = true;
  h->steps = 0;
  return reset_mass(h);
}

int64_t wblbe_step_count(wblbe_handle h) { return h ? h->steps : -1; }

wblbe_status wblbe_set_step_count(wblbe_handle h, int64_t step) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (step < 0) return fail(h, WBLBE_EINVAL, "step must be >= 0");
  h->steps = step;
  return WBLBE_OK;
}
int64_t wblbe_kernel_launches(wblbe_handle h) { return h ? h->launches : -1; }

wblbe_status wblbe_destroy(wblbe_handle h) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  {
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    cudaStreamDestroy(h->capture_stream);
  }
  delete h;
  return WBLBE_OK;
}

const char* wblbe_last_error(wblbe_handle h) { return h ? h->err : g_thread_error; }

size_t wblbe_sequence_scratch_bytes(const wblbe_params* params) {
  if (!params || params->nx < 1 || params->ny < 1) return 0;
  const size_t field = ((size_t)params->nx * params->ny * sizeof(double) + 255) / 256 * 256;
  // two input and two output density fields, then two pairs of stats records
  return 4 * field + 256;
}

}  // extern "C"

namespace {

// Streams, events and the page-locked statistics buffer of one
// wblbe_run_sequence call; released (after the streams drain) on every
// return path.
struct SequenceRes {
  cudaStream_t cin = nullptr, cout = nullptr;
  cudaEvent_t ev[8] = {};
  double* host_rec = nullptr;
  cudaStream_t compute = nullptr;
  ~SequenceRes() {
    if (compute) cudaStreamSynchronize(compute);
    if (cin) {
      cudaStreamSynchronize(cin);
      cudaStreamDestroy(cin);
    }
    if (cout) {
      cudaStreamSynchronize(cout);
      cudaStreamDestroy(cout);
    }
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (host_rec) cudaFreeHost(host_rec);
  }
};

}  // namespace

extern "C" {

wblbe_status wblbe_run_sequence(wblbe_handle h, int32_t n, const double* const* rho_in,
                                int64_t nsteps, double* const* rho_out, wblbe_stats* stats,
                                void* scratch, size_t scratch_bytes) {
  if (!h) return fail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (n < 0 || nsteps < 0) return fail(h, WBLBE_EINVAL, "n and nsteps must be >= 0");
  if (n == 0) return WBLBE_OK;
  if (!rho_in || !rho_out || !scratch) return fail(h, WBLBE_EINVAL, "NULL argument");
  for (int k = 0; k < n; ++k)
    if (!rho_in[k] || !rho_out[k]) return fail(h, WBLBE_EINVAL, "rho_in[%d] or rho_out[%d] is NULL", k, k);
  const size_t need = wblbe_sequence_scratch_bytes(&h->p);
  if (scratch_bytes < need || reinterpret_cast<uintptr_t>(scratch) % 256 != 0)
    return fail(h, WBLBE_EINVAL, "scratch must hold %zu bytes, 256-byte aligned", need);
  DeviceGuard dg(h->device);
  const size_t bytes = (size_t)h->p.nx * h->p.ny * sizeof(double);
  const size_t field = (bytes + 255) / 256 * 256;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  double* in[2] = {reinterpret_cast<double*>(base), reinterpret_cast<double*>(base + field)};
  double* out[2] = {reinterpret_cast<double*>(base + 2 * field),
                    reinterpret_cast<double*>(base + 3 * field)};
  // slot b: [initial-state record, final-state record]
  double* rec = reinterpret_cast<double*>(base + 4 * field);
  constexpr int kPair = 2 * kStatRec;
  static_assert(2 * kPair * sizeof(double) <= 256, "stats records fit the scratch tail");

  SequenceRes r;
  r.compute = h->stream;
  CU(h, cudaStreamCreateWithFlags(&r.cin, cudaStreamNonBlocking));
  CU(h, cudaStreamCreateWithFlags(&r.cout, cudaStreamNonBlocking));
  for (cudaEvent_t& e : r.ev) CU(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEvent_t* ev_in = r.ev;        // input b copied
  cudaEvent_t* ev_used = r.ev + 2;  // input b consumed by the initialisation
  cudaEvent_t* ev_done = r.ev + 4;  // output b and its records written
  cudaEvent_t* ev_out = r.ev + 6;   // output b and its records copied out
  CU(h, cudaHostAlloc(reinterpret_cast<void**>(&r.host_rec), (size_t)n * kPair * sizeof(double),
                      cudaHostAllocDefault));

  auto h2d = [&](int k) -> wblbe_status {
    const int b = k & 1;
    if (k >= 2) CU(h, cudaStreamWaitEvent(r.cin, ev_used[b], 0));
    CU(h, cudaMemcpyAsync(in[b], rho_in[k], bytes, cudaMemcpyHostToDevice, r.cin));
    CU(h, cudaEventRecord(ev_in[b], r.cin));
    return WBLBE_OK;
  };
  wblbe_status st = h2d(0);
  if (st != WBLBE_OK) return st;
  for (int k = 0; k < n; ++k) {
    const int b = k & 1;
    if (k + 1 < n) {
      st = h2d(k + 1);           // overlaps state k's steps
      if (st != WBLBE_OK) return st;
    }
    CU(h, cudaStreamWaitEvent(h->stream, ev_in[b], 0));
    if (k >= 2) CU(h, cudaStreamWaitEvent(h->stream, ev_out[b], 0));
    st = issue_init(h, in[b]);
    if (st != WBLBE_OK) return st;
    CU(h, cudaEventRecord(ev_used[b], h->stream));
    st = run_moments(h, nullptr, nullptr, nullptr, nullptr, rec + b * kPair);
    if (st != WBLBE_OK) return st;
    st = wblbe_step(h, nsteps);
    if (st != WBLBE_OK) return st;
    st = run_moments(h, out[b], nullptr, nullptr, nullptr, rec + b * kPair + kStatRec);
    if (st != WBLBE_OK) return st;
    CU(h, cudaEventRecord(ev_done[b], h->stream));
    // state k's results leave while state k + 1 is computed
    CU(h, cudaStreamWaitEvent(r.cout, ev_done[b], 0));
    CU(h, cudaMemcpyAsync(rho_out[k], out[b], bytes, cudaMemcpyDeviceToHost, r.cout));
    CU(h, cudaMemcpyAsync(r.host_rec + (size_t)k * kPair, rec + b * kPair, kPair * sizeof(double),
                          cudaMemcpyDeviceToHost, r.cout));
    CU(h, cudaEventRecord(ev_out[b], r.cout));
  }
  CU(h, cudaStreamSynchronize(r.cout));
  CU(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < n; ++k) {
    const double* v0 = r.host_rec + (size_t)k * kPair;
    const double* v = v0 + kStatRec;
    if (k == n - 1) h->mass0 = v0[0];   // the handle keeps the last state
    if (!stats) continue;
    wblbe_stats& o = stats[k];
    o.step = nsteps;
    o.mass = v[0];
    o.kinetic = v[1];
    o.umax = v[2];
    o.mu_min = v[3];
    o.mu_max = v[4];
    o.nonfinite = v[5] != 0.0 || !std::isfinite(v[0]);
    o.mass_drift_rel = v0[0] != 0.0 ? (v[0] - v0[0]) / v0[0] : 0.0;
  }
  return WBLBE_OK;
}

}  // extern "C"

// Out-of-bounds accesses that a library built with -DWBLBE_DEBUG_BOUNDS has
// seen (and skipped) on the current device, summed over its kernels;
// 0xFFFFFFFF if the library was built without the checks.
extern "C" unsigned int wblbe_debug_bounds_errors(int32_t reset) {
  const unsigned int a = read_bounds_errors(reset != 0);
  const unsigned int b = batch_bounds_errors(reset != 0);
  const unsigned int c = variants_bounds_errors(reset != 0);
  if (a == 0xFFFFFFFFu || b == 0xFFFFFFFFu || c == 0xFFFFFFFFu) return 0xFFFFFFFFu;
  if (a == 0xFFFFFFFEu || b == 0xFFFFFFFEu || c == 0xFFFFFFFEu) return 0xFFFFFFFEu;
  return a + b + c;
}
