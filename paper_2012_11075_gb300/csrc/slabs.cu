// One lattice split into row slabs: the wblbe_slabs_* half of
// include/wblbe.h.
//
// The update of Eq. D2Q9 is local: a node's new populations depend on the
// populations pulled from its 3 x 3 neighbourhood, on the densities of the
// 5 x 5 neighbourhood (through mu and its gradient, Sec. II) and so on the
// post-collision populations of the 7 x 7 neighbourhood of the previous
// step.  A slab of rows [Y_k, Y_k+1) therefore advances one step from its own
// rows and 3 ghost rows on each side, the neighbouring slabs' rows of the
// previous step; one exchange per step brings them up to date.
//
// Each slab stores its rows with the ghost rows around them, H_k = n_k + 6
// rows (stored row b holds global row Y_k - 3 + b), in the layout of a
// single lattice (nine planes, ping-pong buffers).  A step runs the strip
// kernel of the single-lattice path on the owned rows [3, 3 + n_k) of every
// slab (their stencils reach the ghost rows, never past them), then copies
// each slab's first and last 3 owned rows of the new state into the ghost
// rows of its neighbours (the slabs are periodic: slab 0's lower ghosts come
// from the last slab).  Every node is computed by the same code in the same
// order as in the whole lattice, and the FP32 rounding draws use the global
// row, so results equal the single-lattice run bit for bit.
//
// On one device the slabs' kernels of a step run side by side on forked
// streams (each covers 1/nslabs of the rows, so together they fill the GPU
// as one whole-lattice launch does), then one kernel copies every slab's
// ghost rows; chunks of kSlabGraphSteps steps replay from a captured CUDA
// graph.  The row partition and the exchange plan are what a run across
// devices would also use.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "../../include/wblbe.h"
#include "lbm_kernels.cuh"
#include "strip_launch.cuh"

using namespace wblbe;

namespace {

constexpr int kGhost = 3;                 // ghost rows on each side of a slab
constexpr int kSlabGraphSteps = 16;       // steps per graph replay (even)
constexpr size_t kAlignS = 256;
constexpr int kSlabMomentsRows = 16;

thread_local char g_slabs_error[256] = "";

size_t align_s(size_t v) { return (v + kAlignS - 1) / kAlignS * kAlignS; }

// First global row of slab k of nslabs on ny rows (k = nslabs gives ny).
// Boundaries fall on even rows (the FP32 stochastic rounding pairs rows
// 2j, 2j + 1; see pair_uniforms).
int slab_row(int k, int nslabs, int ny) {
  if (k <= 0) return 0;
  if (k >= nslabs) return ny;
  return (int)(((long long)k * ny / nslabs) & ~1LL);
}

bool slab_params_valid(const wblbe_params* p, int nslabs, char* why, size_t n) {
  if (!p) { snprintf(why, n, "params is NULL"); return false; }
  if (nslabs < 1) { snprintf(why, n, "nslabs must be >= 1"); return false; }
  if (p->nx < 1 || p->ny < 1) { snprintf(why, n, "nx, ny must be >= 1"); return false; }
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) { snprintf(why, n, "tau must be > 0.5"); return false; }
  if (!(p->kappa >= 0.0) || !(p->beta > 0.0)) { snprintf(why, n, "need kappa >= 0, beta > 0"); return false; }
  if (!(p->rho_g > 0.0) || !(p->rho_l > p->rho_g)) { snprintf(why, n, "need rho_l > rho_g > 0"); return false; }
  if (!std::isfinite(p->rho0)) { snprintf(why, n, "rho0 must be finite"); return false; }
  if (p->scheme < WBLBE_STANDARD || p->scheme > WBLBE_STANDARD_TEXTBOOK) {
    snprintf(why, n, "slabs run schemes 0-3 (the E6 variant has its own tile kernel)");
    return false;
  }
  if (p->precision != WBLBE_FP64 && p->precision != WBLBE_FP32_SHIFTED) {
    snprintf(why, n, "unknown precision %d", p->precision); return false;
  }
  if (p->precision == WBLBE_FP32_SHIFTED && std::isinf(p->rho_ref)) {
    snprintf(why, n, "rho_ref must be finite or NaN"); return false;
  }
  for (int k = 0; k < nslabs; ++k)
    if (slab_row(k + 1, nslabs, p->ny) - slab_row(k, nslabs, p->ny) < kGhost) {
      snprintf(why, n, "every slab needs at least %d rows (ny = %d, nslabs = %d)", kGhost,
               p->ny, nslabs);
      return false;
    }
  return true;
}

double slab_rho_ref(const wblbe_params& p) {
  if (p.precision == WBLBE_FP64) return 0.0;
  return std::isnan(p.rho_ref) ? p.rho_g : p.rho_ref;
}

// The stored shift s_i (the scheme's rest equilibrium at rho_ref; 0 in FP64
// apart from the well-balanced rho0 vector).
void slab_shift(const wblbe_params& p, double s[9]) {
  const double w[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
  const double rr = slab_rho_ref(p);
  for (int i = 0; i < 9; ++i)
    s[i] = p.scheme == WBLBE_WELL_BALANCED ? ((i == 0) ? rr - (1.0 - w[0]) * p.rho0 : w[i] * p.rho0)
                                           : w[i] * rr;
}

struct SlabShift {
  double s[9];
};

// Initial state of one slab, ghost rows included: stored row b is global
// row Y = b + y_off (wrapped); P_i(b) = f_i^eq(rho(Y + c_i), u = 0) - s_i.
template <typename T>
__global__ void slab_init_kernel(const double* __restrict__ rho, T* __restrict__ dst, int nx,
                                 int ny, int pitch, long long plane, int y_off, int wb,
                                 double rho0, SlabShift sh) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (x >= nx) return;
  const double w[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int yy = wrap_index(b + y_off + cy[i], ny), xx = wrap_index(x + cx[i], nx);
    const double r = rho[(size_t)yy * nx + xx];
    const double fe = wb ? ((i == 0) ? r - (1.0 - w[0]) * rho0 : w[i] * rho0) : w[i] * r;
    dst[i * plane + (long long)b * pitch + x] = (T)(fe - sh.s[i]);
  }
}

// Populations f_i(x, Y) of direction dir for the slab's owned global rows
// [y_lo, y_lo + n): f_i = P_i(x - c_ix, b - c_iy) + s_i with b = Y - y_off.
template <typename T>
__global__ void slab_get_kernel(const T* __restrict__ src, double* __restrict__ f, int nx,
                                int pitch, long long plane, int y_lo, int y_off, int dir,
                                double shift) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = y_lo + blockIdx.y;
  if (x >= nx) return;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int b = Y - y_off - cy[dir];
  const int xx = wrap_index(x - cx[dir], nx);
  f[(size_t)Y * nx + x] = (double)src[dir * plane + (long long)b * pitch + xx] + shift;
}

}  // namespace

struct wblbe_slabs {
  wblbe_params p;
  int nslabs;
  int device;
  cudaStream_t stream;
  size_t elem;
  int pitch;
  struct Slab {
    int y0, n, H;                // first global row, owned rows, stored rows
    long long plane;             // elements per plane (pitch * H)
    unsigned char* buf[2];
  };
  std::vector<Slab> slabs;
  int cur;
  int tile_x, rows_per_cta;
  std::vector<int> slab_rows;    // rows per CTA of each slab's step launch
  double* stage;                 // nx * ny float64 (host I/O)
  double* partials;
  int max_records;
  double* stats_dev;
  long long* step_dev;           // step of the first step of a graph replay
  void* xdesc;                   // exchange table (XSlab[nslabs]) in the workspace
  std::vector<cudaStream_t> side;  // nslabs - 1 streams for the slabs' kernels
  std::vector<cudaEvent_t> ev;     // fork event, then one join event per side stream
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  int64_t steps, launches;
  double mass0;
  bool have_state;
  char err[256];
};

namespace {

wblbe_status sfail(wblbe_slabs* h, wblbe_status st, const char* fmt, ...) {
  char* dst = h ? h->err : g_slabs_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 256, fmt, ap);
  va_end(ap);
  return st;
}

#define SCU(h, call)                                                           \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return sfail((h), WBLBE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct SlabLayout {
  int pitch;
  size_t elem;
  std::vector<size_t> off_buf;   // 2 per slab
  size_t off_stage, off_partials, off_stats, off_step, off_xdesc, total;
  int max_records;
};

int slab_tile(int nx) { return nx >= 128 ? 128 : (nx > 32 ? 64 : 32); }

// A slab as the exchange kernel sees it.
struct XSlab {
  unsigned char* buf[2];
  long long plane_bytes;         // bytes per population plane
  int n;                         // owned rows
  int pad;
};

SlabLayout slab_layout(const wblbe_params* p, int nslabs) {
  SlabLayout L{};
  L.elem = p->precision == WBLBE_FP64 ? 8 : 4;
  const int align_elems = (int)(128 / L.elem);
  L.pitch = (p->nx + align_elems - 1) / align_elems * align_elems;
  size_t off = 0;
  int records = 0;
  for (int k = 0; k < nslabs; ++k) {
    const int n = slab_row(k + 1, nslabs, p->ny) - slab_row(k, nslabs, p->ny);
    const size_t bytes = align_s((size_t)9 * L.pitch * (n + 2 * kGhost) * L.elem);
    L.off_buf.push_back(off);
    off += bytes;
    L.off_buf.push_back(off);
    off += bytes;
    // records of a moments pass or a step (>= 32 columns, >= 8 rows per CTA)
    records += ((p->nx + 31) / 32) * ((n + 7) / 8);
  }
  L.max_records = records;
  L.off_stage = off; off += align_s((size_t)p->nx * p->ny * sizeof(double));
  L.off_partials = off; off += align_s((size_t)records * kStatRec * sizeof(double));
  L.off_stats = off; off += align_s(8 * sizeof(double));
  L.off_step = off; off += align_s(sizeof(long long));
  L.off_xdesc = off; off += align_s(sizeof(XSlab) * nslabs);
  L.total = off;
  return L;
}

KParams slab_kparams(const wblbe_slabs* h, int k, int rows) {
  const wblbe_params& p = h->p;
  const auto& s = h->slabs[k];
  KParams kp{};
  kp.nx = p.nx;
  kp.ny = s.H;                      // stored rows; the owned ones never wrap
  kp.pitch = h->pitch;
  kp.rows = rows;
  kp.plane = s.plane;
  kp.omega = 1.0 / p.tau;
  kp.kforce = 1.0 - 1.0 / (2.0 * p.tau);
  kp.kappa = p.kappa;
  kp.two_beta = 2.0 * p.beta;
  const double rr = slab_rho_ref(p);
  kp.rho_ref = rr;
  kp.dl = rr - p.rho_l;
  kp.dg = rr - p.rho_g;
  kp.step = h->steps;
  kp.row_lo = kGhost;
  kp.row_hi = kGhost + s.n;
  kp.y_offset = s.y0 - kGhost;
  return kp;
}

cudaError_t slab_launch(const wblbe_slabs* h, int mode, const void* src, void* dst,
                        const KParams& kp, const MomentsOut& mo, int tile,
                        cudaStream_t stream = nullptr) {
  return launch_strip_any(h->p.scheme, h->p.precision == WBLBE_FP64, mode, src, dst, kp, mo,
                          tile, stream ? stream : h->stream);
}

// Ghost rows of every slab's buffer `which` from its neighbours' owned rows,
// in 16-byte pieces (rows are whole multiples of 128 bytes): blockIdx.z is
// the slab; blockIdx.y the side (lower ghosts <- the last 3 owned rows of
// the slab below; upper ghosts <- the first 3 owned rows of the slab above),
// the ghost row and the plane.
__global__ void __launch_bounds__(128)
    slab_exchange_kernel(const XSlab* __restrict__ xs, int nslabs, int which, int row_pieces) {
  const int k = blockIdx.z;
  const int q = blockIdx.y;                 // 0 .. 2 * kGhost * 9 - 1
  const int side = q / (kGhost * 9), r = (q / 9) % kGhost, i = q % 9;
  const XSlab me = xs[k];
  const XSlab nb = xs[side == 0 ? (k + nslabs - 1) % nslabs : (k + 1) % nslabs];
  const long long row_bytes = (long long)row_pieces * 16;
  const int dst_row = side == 0 ? r : kGhost + me.n + r;
  const int src_row = side == 0 ? nb.n + r : kGhost + r;
  const uint4* src = reinterpret_cast<const uint4*>(nb.buf[which] + i * nb.plane_bytes +
                                                    src_row * row_bytes);
  uint4* dst = reinterpret_cast<uint4*>(me.buf[which] + i * me.plane_bytes + dst_row * row_bytes);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < row_pieces; c += gridDim.x * blockDim.x)
    dst[c] = src[c];
}

__global__ void slab_set_step_kernel(long long* dst, long long v) { *dst = v; }

wblbe_status exchange(wblbe_slabs* h, int which, cudaStream_t stream) {
  const int row_pieces = (int)((size_t)h->pitch * h->elem / 16);
  dim3 grid((row_pieces + 127) / 128, 2 * kGhost * 9, h->nslabs);
  slab_exchange_kernel<<<grid, 128, 0, stream>>>(static_cast<const XSlab*>(h->xdesc), h->nslabs,
                                                 which, row_pieces);
  SCU(h, cudaGetLastError());
  return WBLBE_OK;
}

// One step from buffer `from` on `stream`: the slabs' kernels side by side
// (slab 0 on `stream`, slab k on side stream k - 1, forked from and joined
// back into `stream` by events), then the exchange.  The FP32 draws take
// the step t = step + *step_base (step_base may be null).
wblbe_status issue_slab_step(wblbe_slabs* h, int from, cudaStream_t stream, long long step,
                             const long long* step_base) {
  const int S = h->nslabs;
  if (S > 1) {
    SCU(h, cudaEventRecord(h->ev[0], stream));
    for (int k = 1; k < S; ++k) SCU(h, cudaStreamWaitEvent(h->side[k - 1], h->ev[0], 0));
  }
  for (int k = 0; k < S; ++k) {
    KParams kp = slab_kparams(h, k, h->slab_rows[k]);
    kp.step = step;
    kp.step_base = step_base;
    MomentsOut mo{};
    SCU(h, slab_launch(h, kModeStep, h->slabs[k].buf[from], h->slabs[k].buf[1 - from], kp, mo,
                       h->tile_x, k == 0 ? stream : h->side[k - 1]));
  }
  for (int k = 1; k < S; ++k) {
    SCU(h, cudaEventRecord(h->ev[k], h->side[k - 1]));
    SCU(h, cudaStreamWaitEvent(stream, h->ev[k], 0));
  }
  return exchange(h, 1 - from, stream);
}

void drop_slab_graph(wblbe_slabs* h) {
  if (h->graph_valid) cudaGraphExecDestroy(h->graph);
  h->graph_valid = false;
}

// kSlabGraphSteps steps from buffer 0, the steps' indices relative to the
// base word step_dev (set before every replay).
wblbe_status build_slab_graph(wblbe_slabs* h) {
  drop_slab_graph(h);
  cudaGraph_t g = nullptr;
  SCU(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
  wblbe_status st = WBLBE_OK;
  for (int k = 0; k < kSlabGraphSteps && st == WBLBE_OK; ++k)
    st = issue_slab_step(h, k & 1, h->capture_stream, k, h->step_dev);
  cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &g);
  if (st != WBLBE_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st != WBLBE_OK) return st;
    return sfail(h, WBLBE_ECUDA, "slab graph capture: %s", cudaGetErrorString(ce));
  }
  cudaError_t ie = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return sfail(h, WBLBE_ECUDA, "slab graph instantiate: %s", cudaGetErrorString(ie));
  h->graph_valid = true;
  return WBLBE_OK;
}

// Moments of the current state into device fields (may be null) and the
// stats record; every slab reduces its owned rows into its own records.
wblbe_status slab_moments(wblbe_slabs* h, double* rho, double* ux, double* uy, double* mu) {
  const int tile = slab_tile(h->p.nx);
  int rec = 0;
  for (int k = 0; k < h->nslabs; ++k) {
    KParams kp = slab_kparams(h, k, kSlabMomentsRows);
    MomentsOut mo{rho, ux, uy, mu, h->partials + (size_t)rec * kStatRec};
    SCU(h, slab_launch(h, kModeMoments, h->slabs[k].buf[h->cur], nullptr, kp, mo, tile));
    rec += ((h->p.nx + tile - 1) / tile) * ((h->slabs[k].n + kSlabMomentsRows - 1) / kSlabMomentsRows);
  }
  stats_finalize_kernel<<<1, 256, 0, h->stream>>>(h->partials, rec, h->stats_dev);
  SCU(h, cudaGetLastError());
  h->launches += h->nslabs + 1;
  return WBLBE_OK;
}

wblbe_status slab_read_stats(wblbe_slabs* h, wblbe_stats* out) {
  double v[kStatRec];
  SCU(h, cudaMemcpyAsync(v, h->stats_dev, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  SCU(h, cudaStreamSynchronize(h->stream));
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

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DevGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

}  // namespace

extern "C" {

wblbe_status wblbe_slabs_rows(int32_t ny, int32_t nslabs, int32_t* row_starts) {
  if (ny < 1 || nslabs < 1 || !row_starts) return sfail(nullptr, WBLBE_EINVAL, "bad arguments");
  for (int k = 0; k <= nslabs; ++k) row_starts[k] = slab_row(k, nslabs, ny);
  for (int k = 0; k < nslabs; ++k)
    if (row_starts[k + 1] - row_starts[k] < kGhost)
      return sfail(nullptr, WBLBE_EINVAL, "every slab needs at least %d rows", kGhost);
  return WBLBE_OK;
}

size_t wblbe_slabs_workspace_bytes(const wblbe_params* params, int32_t nslabs) {
  char why[256];
  if (!slab_params_valid(params, nslabs, why, sizeof(why))) return 0;
  if ((long long)(params->ny + 6 * nslabs) * ((params->nx + 31) / 32 * 32) >= (1LL << 31)) return 0;
  return slab_layout(params, nslabs).total;
}

wblbe_status wblbe_slabs_create(const wblbe_params* params, int32_t nslabs, void* dev_workspace,
                                size_t workspace_bytes, void* cuda_stream,
                                wblbe_slabs_handle* out) {
  char why[256];
  if (!out) return sfail(nullptr, WBLBE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!slab_params_valid(params, nslabs, why, sizeof(why)))
    return sfail(nullptr, WBLBE_EINVAL, "%s", why);
  const size_t need = wblbe_slabs_workspace_bytes(params, nslabs);
  if (need == 0) return sfail(nullptr, WBLBE_EINVAL, "lattice too large");
  if (!dev_workspace || ((uintptr_t)dev_workspace % kAlignS) != 0)
    return sfail(nullptr, WBLBE_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < need)
    return sfail(nullptr, WBLBE_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
  wblbe_slabs* h = new (std::nothrow) wblbe_slabs();
  if (!h) return sfail(nullptr, WBLBE_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return sfail(nullptr, WBLBE_ECUDA, "no CUDA device");
  }
  {
    // the strip kernels' shared-memory limits (as the single-lattice runtime)
    cudaError_t e = allow_smem_strip_all();
    if (e != cudaSuccess) {
      delete h;
      return sfail(nullptr, WBLBE_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    }
  }
  const SlabLayout L = slab_layout(params, nslabs);
  unsigned char* ws = static_cast<unsigned char*>(dev_workspace);
  h->p = *params;
  h->nslabs = nslabs;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->elem = L.elem;
  h->pitch = L.pitch;
  for (int k = 0; k < nslabs; ++k) {
    wblbe_slabs::Slab s{};
    s.y0 = slab_row(k, nslabs, params->ny);
    s.n = slab_row(k + 1, nslabs, params->ny) - s.y0;
    s.H = s.n + 2 * kGhost;
    s.plane = (long long)L.pitch * s.H;
    s.buf[0] = ws + L.off_buf[2 * k];
    s.buf[1] = ws + L.off_buf[2 * k + 1];
    h->slabs.push_back(s);
  }
  h->stage = reinterpret_cast<double*>(ws + L.off_stage);
  h->partials = reinterpret_cast<double*>(ws + L.off_partials);
  h->max_records = L.max_records;
  h->stats_dev = reinterpret_cast<double*>(ws + L.off_stats);
  h->step_dev = reinterpret_cast<long long*>(ws + L.off_step);
  h->xdesc = ws + L.off_xdesc;
  h->cur = 0;
  {
    // the exchange table, streams and events of the step
    std::vector<XSlab> xs;
    for (const auto& s : h->slabs)
      xs.push_back(XSlab{{s.buf[0], s.buf[1]}, s.plane * (long long)L.elem, s.n, 0});
    cudaError_t e = cudaMemcpy(h->xdesc, xs.data(), xs.size() * sizeof(XSlab),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
    for (int k = 1; k < nslabs && e == cudaSuccess; ++k) {
      cudaStream_t st = nullptr;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) h->side.push_back(st);
    }
    for (int k = 0; k < nslabs && e == cudaSuccess; ++k) {
      cudaEvent_t ev = nullptr;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) h->ev.push_back(ev);
    }
    if (e != cudaSuccess) {
      for (cudaStream_t st : h->side) cudaStreamDestroy(st);
      for (cudaEvent_t ev : h->ev) cudaEventDestroy(ev);
      if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
      delete h;
      return sfail(nullptr, WBLBE_ECUDA, "slab streams: %s", cudaGetErrorString(e));
    }
  }
  // launch shape: 128-column strips, and runs of rows such that the slabs'
  // step launches together make whole resident waves, as the single-lattice
  // default does for the whole lattice: m * B row runs (B = resident CTAs /
  // strips) shared out over the slabs in proportion to their rows, each
  // slab at least one (even rows, at least 8).  m = 1 unless the runs of
  // different slabs would then differ by more than a quarter in length
  // (8 slabs of 512 rows in 23 runs: 172 and 256), which leaves the longest
  // runs running alone at the end of every step; then the fewest waves
  // (up to 4) that bring them within it.
  h->tile_x = slab_tile(params->nx);
  {
    int nsm = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm =
        resident_strip_any(params->scheme, params->precision == WBLBE_FP64, h->tile_x);
    const long long strips = (params->nx + h->tile_x - 1) / h->tile_x;
    const long long B = std::max<long long>((long long)per_sm * nsm / strips, 1);
    std::vector<int> best;
    for (int m = 1; m <= 4; ++m) {
      const long long Bm = std::max<long long>(m * B, nslabs);
      std::vector<long long> segs(nslabs);
      long long total = 0;
      for (int k = 0; k < nslabs; ++k) {
        segs[k] = std::max<long long>(1, (Bm * h->slabs[k].n + params->ny / 2) / params->ny);
        total += segs[k];
      }
      // take runs back from the slabs with the most until the total fits
      while (total > Bm) {
        int kmax = 0;
        for (int k = 1; k < nslabs; ++k)
          if (segs[k] > segs[kmax]) kmax = k;
        if (segs[kmax] <= 1) break;
        --segs[kmax];
        --total;
      }
      std::vector<int> rows_k;
      int lo = 1 << 30, hi = 0;
      for (int k = 0; k < nslabs; ++k) {
        long long rows = (h->slabs[k].n + segs[k] - 1) / segs[k];
        if (rows < 8) rows = 8;
        rows += rows & 1;
        rows_k.push_back((int)rows);
        lo = std::min(lo, (int)rows);
        hi = std::max(hi, (int)rows);
      }
      best = rows_k;
      if (4 * hi <= 5 * lo) break;
    }
    h->slab_rows = best;
    h->rows_per_cta = *std::max_element(best.begin(), best.end());
  }
  *out = h;
  return WBLBE_OK;
}

wblbe_status wblbe_slabs_init_rho(wblbe_slabs_handle h, const double* rho, int32_t rho_on_device) {
  if (!h) return sfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!rho) return sfail(h, WBLBE_EINVAL, "rho is NULL");
  DevGuard dg(h->device);
  const double* src = rho;
  if (!rho_on_device) {
    SCU(h, cudaMemcpyAsync(h->stage, rho, (size_t)h->p.nx * h->p.ny * sizeof(double),
                           cudaMemcpyHostToDevice, h->stream));
    src = h->stage;
  }
  SlabShift sh{};
  slab_shift(h->p, sh.s);
  const int wb = h->p.scheme == WBLBE_WELL_BALANCED;
  h->cur = 0;
  for (const auto& s : h->slabs) {
    dim3 grid((h->p.nx + 127) / 128, s.H);
    if (h->p.precision == WBLBE_FP64)
      slab_init_kernel<double><<<grid, 128, 0, h->stream>>>(
          src, reinterpret_cast<double*>(s.buf[0]), h->p.nx, h->p.ny, h->pitch, s.plane,
          s.y0 - kGhost, wb, h->p.rho0, sh);
    else
      slab_init_kernel<float><<<grid, 128, 0, h->stream>>>(
          src, reinterpret_cast<float*>(s.buf[0]), h->p.nx, h->p.ny, h->pitch, s.plane,
          s.y0 - kGhost, wb, h->p.rho0, sh);
    SCU(h, cudaGetLastError());
    h->launches += 1;
  }
  h->steps = 0;
  h->have_state = true;
  wblbe_status st = slab_moments(h, nullptr, nullptr, nullptr, nullptr);
  if (st != WBLBE_OK) return st;
  wblbe_stats s{};
  st = slab_read_stats(h, &s);
  if (st != WBLBE_OK) return st;
  h->mass0 = s.mass;
  return WBLBE_OK;
}

wblbe_status wblbe_slabs_step(wblbe_slabs_handle h, int64_t nsteps) {
  if (!h) return sfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (nsteps < 0) return sfail(h, WBLBE_EINVAL, "nsteps must be >= 0");
  if (!h->have_state) return sfail(h, WBLBE_EINVAL, "no state: call wblbe_slabs_init_rho first");
  DevGuard dg(h->device);
  const int per_step = h->nslabs + 1;       // the slabs' kernels and the exchange
  auto direct = [&]() -> wblbe_status {
    wblbe_status st = issue_slab_step(h, h->cur, h->stream, h->steps, nullptr);
    if (st != WBLBE_OK) return st;
    h->cur ^= 1;
    h->steps += 1;
    h->launches += per_step;
    return WBLBE_OK;
  };
  int64_t left = nsteps;
  if (left >= kSlabGraphSteps) {
    if (!h->graph_valid) {
      wblbe_status st = build_slab_graph(h);
      if (st != WBLBE_OK) return st;
    }
    // the graph starts from buffer 0
    if (h->cur == 1) {
      wblbe_status st = direct();
      if (st != WBLBE_OK) return st;
      --left;
    }
    while (left >= kSlabGraphSteps) {
      slab_set_step_kernel<<<1, 1, 0, h->stream>>>(h->step_dev, h->steps);
      SCU(h, cudaGetLastError());
      SCU(h, cudaGraphLaunch(h->graph, h->stream));
      h->launches += (int64_t)kSlabGraphSteps * per_step + 1;
      h->steps += kSlabGraphSteps;
      left -= kSlabGraphSteps;
    }
  }
  for (; left > 0; --left) {
    wblbe_status st = direct();
    if (st != WBLBE_OK) return st;
  }
  return WBLBE_OK;
}

wblbe_status wblbe_slabs_moments(wblbe_slabs_handle h, double* rho, double* ux, double* uy,
                                 double* mu, int32_t out_on_device, wblbe_stats* stats) {
  if (!h) return sfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!h->have_state) return sfail(h, WBLBE_EINVAL, "no state: call wblbe_slabs_init_rho first");
  DevGuard dg(h->device);
  wblbe_status st;
  if (out_on_device) {
    st = slab_moments(h, rho, ux, uy, mu);
    if (st != WBLBE_OK) return st;
  } else {
    double* outs[4] = {rho, ux, uy, mu};
    bool any = false;
    const size_t bytes = (size_t)h->p.nx * h->p.ny * sizeof(double);
    for (int q = 0; q < 4; ++q) {
      if (!outs[q]) continue;
      any = true;
      double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
      dev[q] = h->stage;
      st = slab_moments(h, dev[0], dev[1], dev[2], dev[3]);
      if (st != WBLBE_OK) return st;
      SCU(h, cudaMemcpyAsync(outs[q], h->stage, bytes, cudaMemcpyDeviceToHost, h->stream));
    }
    if (!any) {
      st = slab_moments(h, nullptr, nullptr, nullptr, nullptr);
      if (st != WBLBE_OK) return st;
    }
  }
  return slab_read_stats(h, stats);
}

wblbe_status wblbe_slabs_get_populations(wblbe_slabs_handle h, double* f, int32_t on_device) {
  if (!h) return sfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!f) return sfail(h, WBLBE_EINVAL, "f is NULL");
  if (!h->have_state) return sfail(h, WBLBE_EINVAL, "no state: call wblbe_slabs_init_rho first");
  DevGuard dg(h->device);
  double sh[9];
  slab_shift(h->p, sh);
  const size_t field = (size_t)h->p.nx * h->p.ny;
  for (int i = 0; i < 9; ++i) {
    double* dst = on_device ? f + i * field : h->stage;
    for (const auto& s : h->slabs) {
      dim3 grid((h->p.nx + 127) / 128, s.n);
      if (h->p.precision == WBLBE_FP64)
        slab_get_kernel<double><<<grid, 128, 0, h->stream>>>(
            reinterpret_cast<const double*>(s.buf[h->cur]), dst, h->p.nx, h->pitch, s.plane,
            s.y0, s.y0 - kGhost, i, sh[i]);
      else
        slab_get_kernel<float><<<grid, 128, 0, h->stream>>>(
            reinterpret_cast<const float*>(s.buf[h->cur]), dst, h->p.nx, h->pitch, s.plane,
            s.y0, s.y0 - kGhost, i, sh[i]);
      SCU(h, cudaGetLastError());
      h->launches += 1;
    }
    if (!on_device)
      SCU(h, cudaMemcpyAsync(f + i * field, h->stage, field * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
  }
  SCU(h, cudaStreamSynchronize(h->stream));
  return WBLBE_OK;
}

int64_t wblbe_slabs_step_count(wblbe_slabs_handle h) { return h ? h->steps : -1; }
int64_t wblbe_slabs_kernel_launches(wblbe_slabs_handle h) { return h ? h->launches : -1; }

wblbe_status wblbe_slabs_destroy(wblbe_slabs_handle h) {
  if (!h) return sfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  {
    DevGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    drop_slab_graph(h);
    for (cudaStream_t st : h->side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : h->ev) cudaEventDestroy(ev);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  }
  delete h;
  return WBLBE_OK;
}

const char* wblbe_slabs_last_error(wblbe_slabs_handle h) { return h ? h->err : g_slabs_error; }

}  // extern "C"
