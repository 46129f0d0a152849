// Batched, persistent execution of many independent cases (uneven lattice
// sizes and parameters) and the scheduler around it: the wblbe_batch_* half
// of include/wblbe.h.
//
// Device side.  Every resident case owns two population buffers in an arena
// carved from the caller's workspace, stored with ghost columns (see
// strip_pass).  A case is cut into tiles (strips of tile_x columns by
// rows_per_tile rows).  One persistent launch advances every running case by
// K = steps_per_launch lattice steps: its work items are (step j, tile t),
// ordered step-major and claimed with an atomic counter by a fixed grid of
// resident CTAs.  Item (j, t) may start once tile t itself and every tile
// whose data its halo reads (3 nodes: pull + density halo) have finished step
// j - 1 (consecutive steps of one tile may run on different CTAs); each tile
// publishes its finished step in a counter (release/acquire).  Because items
// are claimed in dependency order, the earliest unfinished item always has
// its inputs ready, so the schedule cannot deadlock whatever the number of
// CTAs resident.  Waits are bounded: a wait that runs out sets a status word,
// every CTA stops, and the host reports WBLBE_ETIMEOUT.  The last step of a
// launch also reduces per-tile statistics; a finish kernel folds them per
// case (fixed order) and flips the case's buffer parity.
//
// Host side.  Admission checks a free case slot, arena space for the case
// (first fit) and room in the tile table; the tile table of the running cases
// and the launch descriptor live in device memory, so one captured CUDA graph
// (counter resets + persistent kernel + finish kernel) serves every active
// set.  After each group of launches the host reads the per-case statistics
// and retires converged, exhausted or unstable cases from the running set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/wblbe.h"
#include "lbm_kernels.cuh"

using namespace wblbe;

namespace {

constexpr int kMaxNb = 12;               // neighbour tiles a tile may wait on
static_assert(kMaxNb + 1 <= 32, "one lane of warp 0 per awaited counter");
constexpr int kHaloReach = 3;            // nodes a step reads around its tile
constexpr size_t kAlignB = 256;
constexpr long long kDefaultSpins = 1LL << 22;   // x ~64 ns sleep: about 0.3 s

struct CaseDev {
  KParams kp;
  long long off[2];      // element offsets of the two buffers in the arena
  int cur;               // buffer holding the state
  int pad;
};

struct TileDev {
  int c, x0, y0, y1;
  int nb[kMaxNb];
};

struct RunCase {          // a running case and its tile range
  int c, t0, nt, pad;
};

struct BatchDesc {
  int ntiles, steps, nrun, pad;
};

struct BatchDev {
  void* arena;
  const CaseDev* cases;
  const TileDev* tiles;
  int* done;
  int* head;
  int* status;
  double* tile_stats;
  const BatchDesc* desc;
  long long spins;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T, bool WB, int TX>
__global__ void __launch_bounds__(TX, Staging<T>::min_blocks_batch(TX))
    batch_persistent_kernel(const BatchDev d) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_item, s_ok;
  const int ntiles = d.desc->ntiles, K = d.desc->steps;
  const int total = ntiles * K;
  T* arena = static_cast<T*>(d.arena);
  for (;;) {
    __syncthreads();                       // s_item / s_ok are reused
    if (threadIdx.x == 0) s_item = atomicAdd(d.head, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int j = item / ntiles, t = item - j * ntiles;
    const TileDev tile = d.tiles[t];
    if (threadIdx.x < 32) {
      // warp 0 waits for the tile itself (its step j-1 may run on another
      // CTA) and for every neighbour its halo reads, one counter per lane,
      // so that the waits overlap
      const int lane = threadIdx.x;
      int ok = ld_acquire(d.status) == 0;
      const int nb =
          j == 0 ? -1 : (lane == 0 ? t : (lane <= kMaxNb ? d.tiles[t].nb[lane - 1] : -1));
      if (ok && nb >= 0) {
        long long n = 0;
        while (ld_acquire(d.done + nb) < j) {
          if (++n > d.spins || (n % 256 == 0 && ld_acquire(d.status) != 0)) {
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      ok = __all_sync(0xffffffffu, ok);
      if (lane == 0) {
        if (!ok) atomicOr(d.status, 1);
        s_ok = ok;
      }
    }
    __syncthreads();
    if (!s_ok) break;                      // nothing of this CTA is in flight
    const CaseDev& cs = d.cases[tile.c];
    // the case's parameters in shared memory: no registers held for them,
    // and no reloads after the population stores (which could alias
    // device memory)
    __shared__ KParams s_kp;
    if (threadIdx.x == 0) {
      s_kp = cs.kp;
      s_kp.step += j;                      // the case's time step of this item
    }
    __syncthreads();
    const KParams& kp = s_kp;
    const int cur = (cs.cur + j) & 1;
    const T* src = arena + cs.off[cur];
    T* dst = arena + cs.off[cur ^ 1];
    const MomentsOut mo{};
    constexpr int SCH = WB ? kSchWB : kSchStandard;
    if (j == K - 1)
      strip_pass<T, SCH, kModeStepStats, TX, true>(src, dst, kp, mo, tile.x0, tile.y0, tile.y1,
                                                   d.tile_stats + (size_t)t * kStatRec, smem_raw);
    else
      strip_pass<T, SCH, kModeStep, TX, true>(src, dst, kp, mo, tile.x0, tile.y0, tile.y1,
                                              nullptr, smem_raw);
    __threadfence();                       // this thread's stores, device-wide
    __syncthreads();
    if (threadIdx.x == 0) st_release(d.done + t, j + 1);
  }
}

// Per running case: fold its tile statistics (fixed order) and flip the
// buffer parity by the launch's step count.
__global__ void __launch_bounds__(128)
    batch_finish_kernel(const BatchDev d, CaseDev* cases, const RunCase* run,
                        double* case_stats) {
  __shared__ double red[128][kStatRec];
  const int r = blockIdx.x;
  if (r >= d.desc->nrun) return;
  const RunCase rc = run[r];
  double v[kStatRec] = {0.0, 0.0, 0.0, 1e300, -1e300, 0.0};
  for (int k = threadIdx.x; k < rc.nt; k += blockDim.x) {
    const double* s = d.tile_stats + (size_t)(rc.t0 + k) * kStatRec;
    v[0] += s[0];
    v[1] += s[1];
    v[2] = fmax(v[2], s[2]);
    v[3] = fmin(v[3], s[3]);
    v[4] = fmax(v[4], s[4]);
    v[5] = fmax(v[5], s[5]);
  }
#pragma unroll
  for (int q = 0; q < kStatRec; ++q) red[threadIdx.x][q] = v[q];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double* a = red[threadIdx.x];
      const double* b = red[threadIdx.x + s];
      a[0] += b[0];
      a[1] += b[1];
      a[2] = fmax(a[2], b[2]);
      a[3] = fmin(a[3], b[3]);
      a[4] = fmax(a[4], b[4]);
      a[5] = fmax(a[5], b[5]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* out = case_stats + (size_t)rc.c * kStatRec;
    out[0] = red[0][0];
    out[1] = red[0][1];
    out[2] = sqrt(red[0][2]);
    out[3] = red[0][3];
    out[4] = red[0][4];
    out[5] = red[0][5];
    cases[rc.c].cur ^= (d.desc->steps & 1);
    cases[rc.c].kp.step += d.desc->steps;
  }
}

// Moments of one case (ghost layout), one CTA per tile of the case's grid.
template <typename T, bool WB, int TX>
__global__ void __launch_bounds__(TX, Staging<T>::min_blocks_batch(TX))
    batch_case_moments_kernel(const T* __restrict__ pops, const KParams kp,
                              const MomentsOut mo) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int x0 = blockIdx.x * TX;
  const int y0 = blockIdx.y * kp.rows;
  const int y1 = min(y0 + kp.rows, kp.ny);
  double* rec = mo.partials + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kStatRec;
  constexpr int SCH = WB ? kSchWB : kSchStandard;
  strip_pass<T, SCH, kModeMoments, TX, true>(pops, nullptr, kp, mo, x0, y0, y1, rec, smem_raw);
}

// Initial state of one case in the ghost layout: P_i(x) = f_i^eq(rho(x+c_i), 0)
// - s_i at storage offset x + ghost_off, for every stored column x = -4 ..
// nx + 3 (ghosts included).
template <typename T>
__global__ void batch_init_kernel(const double* __restrict__ rho, T* __restrict__ dst,
                                  int nx, int ny, int pitch, long long plane, int wb,
                                  double rho0, LayoutParams lp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;   // column k - 4
  const int y = blockIdx.y;
  if (k >= nx + 2 * kPad) return;
  const int x = wrap_index(k - kPad, nx);
  const int o = k - kPad + ghost_off<T>();                // storage column
  const double w[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double r = rho[(size_t)wrap_index(y + kCy[i], ny) * nx + wrap_index(x + kCx[i], nx)];
    const double fe = wb ? ((i == 0) ? r - (1.0 - w[0]) * rho0 : w[i] * rho0) : w[i] * r;
    dst[i * plane + (long long)y * pitch + o] = (T)(fe - lp.shift[i]);
  }
}

// f[i][y][x] = P_i(x - c_i) + s_i from the ghost layout (float64 out).
template <typename T>
__global__ void batch_get_pops_kernel(const T* __restrict__ src, double* __restrict__ f, int nx,
                                      int ny, int pitch, long long plane, LayoutParams lp,
                                      int dir) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const int sy = wrap_index(y - kCy[dir], ny);
  const double v =
      (double)src[dir * plane + (long long)sy * pitch + (x - kCx[dir] + ghost_off<T>())];
  f[(size_t)y * nx + x] = v + lp.shift[dir];
}

size_t align_b(size_t v) { return (v + kAlignB - 1) / kAlignB * kAlignB; }

thread_local char g_batch_error[256] = "";

}  // namespace

struct wblbe_batch {
  int scheme, precision;
  size_t elem;
  int max_cases, max_tiles;
  long long max_case_nodes;
  int device;
  cudaStream_t stream, capture_stream;
  unsigned char* ws;
  size_t ws_bytes;
  // control region (device)
  CaseDev* d_cases;
  TileDev* d_tiles;
  RunCase* d_run;
  int* d_done;
  int* d_head;
  int* d_status;
  BatchDesc* d_desc;
  double* d_tile_stats;
  double* d_case_stats;
  double* d_partials;
  double* d_stage;
  unsigned char* arena;
  size_t arena_bytes;
  std::map<size_t, size_t> free_ranges;   // offset -> length (bytes), arena
  struct Case {
    bool used = false, running = false, reported = true;
    int32_t state = WBLBE_CASE_RUNNING;
    wblbe_params p{};
    int pitch = 0;
    long long plane = 0;
    size_t off = 0, bytes = 0;             // arena range (bytes)
    double tol = 0.0;
    int64_t max_steps = 0, steps = 0;
    int cur = 0;
    double mass0 = 0.0;
    wblbe_stats last{};
    int64_t id = -1;
    std::vector<TileDev> tiles;            // local tiles, nb = local indices
    int tiles_tx = 0, tiles_rows = 0;      // configuration they were cut for
  };
  std::vector<Case> cases;
  int64_t next_id = 0;
  wblbe_batch_config cfg{};
  long long spins = kDefaultSpins;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  bool tiles_dirty = true;
  int ntiles = 0, nrun = 0;
  std::vector<RunCase> run_host;
  std::vector<CaseDev> case_host;         // staging of the case table upload
  int64_t launches = 0;
  char err[256] = "";
};

namespace {

wblbe_status bfail(wblbe_batch* b, wblbe_status st, const char* fmt, ...) {
  char* dst = b ? b->err : g_batch_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 256, fmt, ap);
  va_end(ap);
  return st;
}

#define BCU(b, call)                                                            \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return bfail((b), WBLBE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct Control {
  size_t cases, tiles, run, done, head, status, desc, tile_stats, case_stats, partials, stage,
      total;
};

Control control_layout(int max_cases, int max_tiles, long long max_case_nodes) {
  Control c{};
  size_t off = 0;
  c.cases = off; off += align_b(sizeof(CaseDev) * max_cases);
  c.tiles = off; off += align_b(sizeof(TileDev) * max_tiles);
  c.run = off; off += align_b(sizeof(RunCase) * max_cases);
  c.done = off; off += align_b(sizeof(int) * max_tiles);
  c.head = off; off += align_b(sizeof(int));
  c.status = off; off += align_b(sizeof(int));
  c.desc = off; off += align_b(sizeof(BatchDesc));
  c.tile_stats = off; off += align_b(sizeof(double) * kStatRec * max_tiles);
  c.case_stats = off; off += align_b(sizeof(double) * kStatRec * (max_cases + 1));  // +1: scratch
  // per-case moments records: at most ceil(nx/32) * ceil(ny/8) CTAs
  c.partials = off; off += align_b(sizeof(double) * kStatRec * (size_t)(max_case_nodes / 64 + 4096));
  c.stage = off; off += align_b(sizeof(double) * (size_t)max_case_nodes);
  c.total = off;
  return c;
}

int case_pitch(int nx, size_t elem) {
  const int align_elems = (int)(128 / elem);
  const int off = elem == 4 ? ghost_off<float>() : ghost_off<double>();
  // leading offset, right ghosts and chunk overrun
  return (nx + off + 8 + align_elems - 1) / align_elems * align_elems;
}

size_t case_bytes(const wblbe_params* p, size_t elem) {
  const long long plane = (long long)case_pitch(p->nx, elem) * p->ny;
  return 2 * align_b((size_t)9 * plane * elem);
}

bool batch_params_valid(const wblbe_batch* b, const wblbe_params* p, char* why, size_t n) {
  if (!p) { snprintf(why, n, "params is NULL"); return false; }
  if (p->nx < 8 || p->ny < 8) { snprintf(why, n, "batched cases need nx, ny >= 8"); return false; }
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) { snprintf(why, n, "tau must be > 0.5"); return false; }
  if (!(p->kappa >= 0.0) || !(p->beta > 0.0)) { snprintf(why, n, "need kappa >= 0, beta > 0"); return false; }
  if (!(p->rho_g > 0.0) || !(p->rho_l > p->rho_g)) { snprintf(why, n, "need rho_l > rho_g > 0"); return false; }
  if (p->scheme != b->scheme || p->precision != b->precision) {
    snprintf(why, n, "scheme and precision must match the batch"); return false;
  }
  if ((long long)p->nx * p->ny > b->max_case_nodes) {
    snprintf(why, n, "case has %lld nodes, the batch was created for at most %lld",
             (long long)p->nx * p->ny, b->max_case_nodes);
    return false;
  }
  if ((long long)case_pitch(p->nx, b->elem) * p->ny >= (1LL << 31)) {
    snprintf(why, n, "case too large: plane offsets are 32-bit");
    return false;
  }
  return true;
}

// FP32 shift density, as for a single lattice: by default the gas density
double batch_rho_ref(const wblbe_params& p) {
  if (p.precision == WBLBE_FP64) return 0.0;
  return std::isnan(p.rho_ref) ? p.rho_g : p.rho_ref;
}

KParams case_kparams(const wblbe_batch::Case& c, int rows) {
  const wblbe_params& p = c.p;
  KParams k{};
  k.nx = p.nx;
  k.ny = p.ny;
  k.pitch = c.pitch;
  k.rows = rows;
  k.plane = c.plane;
  k.omega = 1.0 / p.tau;
  k.kforce = 1.0 - 1.0 / (2.0 * p.tau);
  k.kappa = p.kappa;
  k.two_beta = 2.0 * p.beta;
  const double rr = batch_rho_ref(p);
  k.rho_ref = rr;
  k.dl = rr - p.rho_l;
  k.dg = rr - p.rho_g;
  k.step = c.steps;                        // advanced on the device by each launch
  k.row_lo = 0;
  k.row_hi = p.ny;
  k.y_offset = 0;
  return k;
}

LayoutParams case_layout(const wblbe_batch::Case& c) {
  LayoutParams lp{};
  lp.nx = c.p.nx;
  lp.ny = c.p.ny;
  lp.pitch = c.pitch;
  lp.plane = c.plane;
  lp.wb = c.p.scheme == WBLBE_WELL_BALANCED;
  lp.rho0 = c.p.rho0;
  const double w[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
  const double rr = batch_rho_ref(c.p);
  // the rest equilibrium at rho_ref (0 in FP64); it carries the WB rho0
  // vector in both precisions, so the kernel never sees rho0
  for (int i = 0; i < 9; ++i) {
    if (lp.wb) lp.shift[i] = (i == 0) ? rr - (1.0 - w[0]) * c.p.rho0 : w[i] * c.p.rho0;
    else lp.shift[i] = w[i] * rr;
  }
  return lp;
}

// Does the periodic interval [a - h, b + h) (mod n) meet [c, d) (0 <= c < d <= n)?
bool periodic_meet(int a, int b, int c, int d, int h, int n) {
  const int len = (b - a) + 2 * h;
  if (len >= n) return true;
  const int s = (((a - h) % n) + n) % n;
  if (s + len <= n) return std::max(s, c) < std::min(s + len, d);
  return std::max(s, c) < d || c < s + len - n;     // [s, n) and [0, s + len - n)
}

// Tiles of a case: strips of tile_x columns (x0 a multiple of tile_x) and
// near-equal runs of about rows_per_tile rows.
void case_tiles(const wblbe_batch::Case& c, int case_idx, const wblbe_batch_config& cfg,
                std::vector<TileDev>& out) {
  const int nx = c.p.nx, ny = c.p.ny;
  const int nseg = std::max(1, ny / std::max(cfg.rows_per_tile, 4));
  // run boundaries on even rows (the FP32 stochastic rounding draws one hash
  // per pair of rows 2j, 2j + 1; see pair_uniforms)
  auto bound = [&](int s) { return s >= nseg ? ny : (int)((long long)s * ny / nseg) & ~1; };
  for (int s = 0; s < nseg; ++s) {
    const int y0 = bound(s), y1 = bound(s + 1);
    for (int x0 = 0; x0 < nx; x0 += cfg.tile_x) {
      TileDev t{};
      t.c = case_idx;
      t.x0 = x0;
      t.y0 = y0;
      t.y1 = y1;
      for (int q = 0; q < kMaxNb; ++q) t.nb[q] = -1;
      out.push_back(t);
    }
  }
}

// Cut a case into tiles for the current configuration and find, for every
// tile, the tiles of the same case its halo reads (local indices).  Cached
// until the configuration changes.
wblbe_status ensure_case_tiles(wblbe_batch* b, wblbe_batch::Case& c) {
  if (c.tiles_tx == b->cfg.tile_x && c.tiles_rows == b->cfg.rows_per_tile && !c.tiles.empty())
    return WBLBE_OK;
  c.tiles.clear();
  case_tiles(c, 0, b->cfg, c.tiles);
  const int nt = (int)c.tiles.size();
  for (int a = 0; a < nt; ++a) {
    TileDev& ta = c.tiles[a];
    const int wa = std::min(b->cfg.tile_x, c.p.nx - ta.x0);
    int n = 0;
    for (int q = 0; q < nt; ++q) {
      if (q == a) continue;
      const TileDev& tq = c.tiles[q];
      const int wq = std::min(b->cfg.tile_x, c.p.nx - tq.x0);
      if (periodic_meet(ta.x0, ta.x0 + wa, tq.x0, tq.x0 + wq, kHaloReach, c.p.nx) &&
          periodic_meet(ta.y0, ta.y1, tq.y0, tq.y1, kHaloReach, c.p.ny)) {
        if (n == kMaxNb) {
          c.tiles.clear();
          return bfail(b, WBLBE_EINVAL, "a tile of case %lld has more than %d neighbours; "
                       "use larger tiles", (long long)c.id, kMaxNb);
        }
        ta.nb[n++] = q;
      }
    }
  }
  c.tiles_tx = b->cfg.tile_x;
  c.tiles_rows = b->cfg.rows_per_tile;
  return WBLBE_OK;
}

wblbe_status upload_case_entry(wblbe_batch* b, int ci) {
  const auto& c = b->cases[ci];
  CaseDev cd{};
  cd.kp = case_kparams(c, b->cfg.rows_per_tile);
  cd.off[0] = (long long)(c.off / b->elem);
  cd.off[1] = (long long)((c.off + c.bytes / 2) / b->elem);
  cd.cur = c.cur;
  BCU(b, cudaMemcpyAsync(b->d_cases + ci, &cd, sizeof(cd), cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));    // cd lives on this stack frame
  return WBLBE_OK;
}

// Concatenate the running cases' tiles (global neighbour indices) and upload
// the tile table and the running-case list.
wblbe_status rebuild_tiles(wblbe_batch* b) {
  std::vector<TileDev> tiles;
  b->run_host.clear();
  for (size_t ci = 0; ci < b->cases.size(); ++ci) {
    auto& c = b->cases[ci];
    if (!c.used || !c.running) continue;
    wblbe_status st = ensure_case_tiles(b, c);
    if (st != WBLBE_OK) return st;
    RunCase rc{};
    rc.c = (int)ci;
    rc.t0 = (int)tiles.size();
    rc.nt = (int)c.tiles.size();
    for (TileDev t : c.tiles) {
      t.c = (int)ci;
      for (int q = 0; q < kMaxNb; ++q)
        if (t.nb[q] >= 0) t.nb[q] += rc.t0;
      tiles.push_back(t);
    }
    b->run_host.push_back(rc);
  }
  if ((int)tiles.size() > b->max_tiles)
    return bfail(b, WBLBE_ENOMEM, "running cases need %zu tiles, the batch holds %d", tiles.size(),
                 b->max_tiles);
  b->ntiles = (int)tiles.size();
  b->nrun = (int)b->run_host.size();
  if (!tiles.empty())
    BCU(b, cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(TileDev),
                           cudaMemcpyHostToDevice, b->stream));
  if (!b->run_host.empty())
    BCU(b, cudaMemcpyAsync(b->d_run, b->run_host.data(), b->run_host.size() * sizeof(RunCase),
                           cudaMemcpyHostToDevice, b->stream));
  // the case table carries rows_per_tile (moments) and the buffer parity:
  // one copy of the whole table (entries of unused slots are never read)
  b->case_host.assign(b->cases.size(), CaseDev{});
  for (size_t ci = 0; ci < b->cases.size(); ++ci) {
    const auto& c = b->cases[ci];
    if (!c.used) continue;
    CaseDev& cd = b->case_host[ci];
    cd.kp = case_kparams(c, b->cfg.rows_per_tile);
    cd.off[0] = (long long)(c.off / b->elem);
    cd.off[1] = (long long)((c.off + c.bytes / 2) / b->elem);
    cd.cur = c.cur;
  }
  if (!b->case_host.empty())
    BCU(b, cudaMemcpyAsync(b->d_cases, b->case_host.data(), b->case_host.size() * sizeof(CaseDev),
                           cudaMemcpyHostToDevice, b->stream));
  // the host buffers above must stay valid until the copies ran
  BCU(b, cudaStreamSynchronize(b->stream));
  b->tiles_dirty = false;
  return WBLBE_OK;
}

template <typename T, bool WB, int TX>
cudaError_t batch_launch_tx(const BatchDev& d, int grid, cudaStream_t s) {
  const size_t smem = strip_smem_bytes(TX, Staging<T>::kStages, sizeof(T));
  batch_persistent_kernel<T, WB, TX><<<grid, TX, smem, s>>>(d);
  return cudaGetLastError();
}

// Resident CTAs of the persistent kernel (sets its shared-memory limit).
template <typename T, bool WB, int TX>
int batch_grid_tx() {
  const size_t smem = strip_smem_bytes(TX, Staging<T>::kStages, sizeof(T));
  cudaFuncSetAttribute(batch_persistent_kernel<T, WB, TX>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<T, WB, TX>, TX,
                                                smem);
  return std::max(1, per_sm) * std::max(1, nsm);
}

template <typename T, bool WB>
int batch_grid(int tile) {
  switch (tile) {
    case 32: return batch_grid_tx<T, WB, 32>();
    case 64: return batch_grid_tx<T, WB, 64>();
    case 128: return batch_grid_tx<T, WB, 128>();
    default: return batch_grid_tx<T, WB, 256>();
  }
}

template <typename T, bool WB>
cudaError_t batch_launch(const BatchDev& d, int tile, int grid, cudaStream_t s) {
  switch (tile) {
    case 32: return batch_launch_tx<T, WB, 32>(d, grid, s);
    case 64: return batch_launch_tx<T, WB, 64>(d, grid, s);
    case 128: return batch_launch_tx<T, WB, 128>(d, grid, s);
    case 256: return batch_launch_tx<T, WB, 256>(d, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

BatchDev batch_dev(const wblbe_batch* b) {
  BatchDev d{};
  d.arena = b->arena;
  d.cases = b->d_cases;
  d.tiles = b->d_tiles;
  d.done = b->d_done;
  d.head = b->d_head;
  d.status = b->d_status;
  d.tile_stats = b->d_tile_stats;
  d.desc = b->d_desc;
  d.spins = b->spins;
  return d;
}

// One persistent launch: reset counters, advance, fold statistics.
cudaError_t issue_launch(wblbe_batch* b, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_done, 0, sizeof(int) * b->max_tiles, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_head, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const BatchDev d = batch_dev(b);
  const bool wb = b->scheme == WBLBE_WELL_BALANCED;
  if (b->precision == WBLBE_FP64)
    e = wb ? batch_launch<double, true>(d, b->cfg.tile_x, grid, s)
           : batch_launch<double, false>(d, b->cfg.tile_x, grid, s);
  else
    e = wb ? batch_launch<float, true>(d, b->cfg.tile_x, grid, s)
           : batch_launch<float, false>(d, b->cfg.tile_x, grid, s);
  if (e != cudaSuccess) return e;
  batch_finish_kernel<<<b->max_cases, 128, 0, s>>>(d, b->d_cases, b->d_run, b->d_case_stats);
  return cudaGetLastError();
}

void drop_batch_graph(wblbe_batch* b) {
  if (b->graph_valid) cudaGraphExecDestroy(b->graph);
  b->graph_valid = false;
}

wblbe_status build_batch_graph(wblbe_batch* b) {
  drop_batch_graph(b);
  // attributes and occupancy queries outside the capture
  const bool wb = b->scheme == WBLBE_WELL_BALANCED;
  const int grid = b->precision == WBLBE_FP64
                       ? (wb ? batch_grid<double, true>(b->cfg.tile_x) : batch_grid<double, false>(b->cfg.tile_x))
                       : (wb ? batch_grid<float, true>(b->cfg.tile_x) : batch_grid<float, false>(b->cfg.tile_x));
  BCU(b, cudaGetLastError());
  cudaGraph_t g = nullptr;
  BCU(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = issue_launch(b, grid, b->capture_stream);
  cudaError_t ce = cudaStreamEndCapture(b->capture_stream, &g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, WBLBE_ECUDA, "batch graph capture: %s",
                 cudaGetErrorString(le != cudaSuccess ? le : ce));
  }
  cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return bfail(b, WBLBE_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(ie));
  b->graph_valid = true;
  return WBLBE_OK;
}

bool alloc_range(wblbe_batch* b, size_t bytes, size_t* off) {
  for (auto it = b->free_ranges.begin(); it != b->free_ranges.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t roff = it->first + bytes;
      b->free_ranges.erase(it);
      if (rest > 0) b->free_ranges[roff] = rest;
      return true;
    }
  }
  return false;
}

void free_range(wblbe_batch* b, size_t off, size_t bytes) {
  auto it = b->free_ranges.emplace(off, bytes).first;
  auto next = std::next(it);
  if (next != b->free_ranges.end() && it->first + it->second == next->first) {
    it->second += next->second;
    b->free_ranges.erase(next);
  }
  if (it != b->free_ranges.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      b->free_ranges.erase(it);
    }
  }
}

// Stats record after the per-case ones, used by single-case moment passes.
double* scratch_stats(const wblbe_batch* b) { return b->d_case_stats + (size_t)b->max_cases * kStatRec; }

int find_case(const wblbe_batch* b, int64_t id) {
  for (size_t i = 0; i < b->cases.size(); ++i)
    if (b->cases[i].used && b->cases[i].id == id) return (int)i;
  return -1;
}

template <typename T, bool WB, int TX>
cudaError_t case_moments_tx(const wblbe_batch* b, const wblbe_batch::Case& c, const MomentsOut& mo,
                            int rows) {
  const size_t smem = strip_smem_bytes(TX, Staging<T>::kStages, sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(batch_case_moments_kernel<T, WB, TX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  KParams kp = case_kparams(c, rows);
  dim3 grid((c.p.nx + TX - 1) / TX, (c.p.ny + rows - 1) / rows);
  const T* pops = reinterpret_cast<const T*>(b->arena + c.off + (c.cur ? c.bytes / 2 : 0));
  batch_case_moments_kernel<T, WB, TX><<<grid, TX, smem, b->stream>>>(pops, kp, mo);
  return cudaGetLastError();
}

// Moments of one case into device fields (may be null) and its stats record.
wblbe_status case_moments(wblbe_batch* b, const wblbe_batch::Case& c, double* rho, double* ux,
                          double* uy, double* mu, double* stats6) {
  const int rows = 16;
  MomentsOut mo{rho, ux, uy, mu, b->d_partials};
  const bool wb = b->scheme == WBLBE_WELL_BALANCED;
  cudaError_t e = b->precision == WBLBE_FP64
                      ? (wb ? case_moments_tx<double, true, 64>(b, c, mo, rows)
                            : case_moments_tx<double, false, 64>(b, c, mo, rows))
                      : (wb ? case_moments_tx<float, true, 64>(b, c, mo, rows)
                            : case_moments_tx<float, false, 64>(b, c, mo, rows));
  if (e != cudaSuccess) return bfail(b, WBLBE_ECUDA, "case moments: %s", cudaGetErrorString(e));
  const int n = ((c.p.nx + 63) / 64) * ((c.p.ny + rows - 1) / rows);
  stats_finalize_kernel<<<1, 256, 0, b->stream>>>(b->d_partials, n, scratch_stats(b));
  (void)stats6;
  BCU(b, cudaGetLastError());
  return WBLBE_OK;
}

// Device part of an admission: the initial state f = f^eq(rho, 0) of case
// slot from the host field rho, its case-table entry and its initial mass.
wblbe_status admit_device(wblbe_batch* b, int slot, const double* rho) {
  wblbe_batch::Case& c = b->cases[slot];
  const wblbe_params& p = c.p;
  const size_t nodes = (size_t)p.nx * p.ny;
  BCU(b, cudaMemcpyAsync(b->d_stage, rho, nodes * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  LayoutParams lp = case_layout(c);
  dim3 grid((p.nx + 2 * kPad + 127) / 128, p.ny);
  const int wb = p.scheme == WBLBE_WELL_BALANCED;
  if (b->precision == WBLBE_FP64)
    batch_init_kernel<double><<<grid, 128, 0, b->stream>>>(
        b->d_stage, reinterpret_cast<double*>(b->arena + c.off), p.nx, p.ny, c.pitch, c.plane,
        wb, p.rho0, lp);
  else
    batch_init_kernel<float><<<grid, 128, 0, b->stream>>>(
        b->d_stage, reinterpret_cast<float*>(b->arena + c.off), p.nx, p.ny, c.pitch, c.plane,
        wb, p.rho0, lp);
  BCU(b, cudaGetLastError());
  wblbe_status st = upload_case_entry(b, slot);
  if (st != WBLBE_OK) return st;
  st = case_moments(b, c, nullptr, nullptr, nullptr, nullptr, nullptr);
  if (st != WBLBE_OK) return st;
  double v[kStatRec];
  BCU(b, cudaMemcpyAsync(v, scratch_stats(b), sizeof(v), cudaMemcpyDeviceToHost, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  c.mass0 = v[0];
  return WBLBE_OK;
}

}  // namespace

extern "C" {

size_t wblbe_batch_workspace_bytes(int32_t max_cases, int32_t max_tiles,
                                   int64_t max_case_nodes, size_t arena_bytes) {
  if (max_cases < 1 || max_tiles < 1 || max_case_nodes < 64) return 0;
  return control_layout(max_cases, max_tiles, max_case_nodes).total + align_b(arena_bytes);
}

size_t wblbe_batch_case_bytes(const wblbe_params* params) {
  if (!params || params->nx < 8 || params->ny < 8) return 0;
  return case_bytes(params, params->precision == WBLBE_FP64 ? 8 : 4);
}

wblbe_status wblbe_batch_create(int32_t scheme, int32_t precision, int32_t max_cases,
                                int32_t max_tiles, int64_t max_case_nodes, void* dev_workspace,
                                size_t workspace_bytes, void* cuda_stream,
                                const wblbe_batch_config* config, wblbe_batch_handle* out) {
  if (!out) return bfail(nullptr, WBLBE_EINVAL, "out is NULL");
  *out = nullptr;
  if (scheme != WBLBE_STANDARD && scheme != WBLBE_WELL_BALANCED)
    return bfail(nullptr, WBLBE_EINVAL,
                 "the batch runs the standard and well-balanced schemes only "
                 "(the comparison variants run on single lattices)");
  if (precision != WBLBE_FP64 && precision != WBLBE_FP32_SHIFTED)
    return bfail(nullptr, WBLBE_EINVAL, "unknown precision");
  if (max_cases < 1 || max_tiles < 1 || max_case_nodes < 64)
    return bfail(nullptr, WBLBE_EINVAL, "need max_cases, max_tiles >= 1, max_case_nodes >= 64");
  if (!config || (config->tile_x != 32 && config->tile_x != 64 && config->tile_x != 128 &&
                  config->tile_x != 256) ||
      config->rows_per_tile < 4 || config->steps_per_launch < 1)
    return bfail(nullptr, WBLBE_EINVAL, "config: tile_x 32/64/128/256, rows_per_tile >= 4, steps >= 1");
  const Control ctl = control_layout(max_cases, max_tiles, max_case_nodes);
  if (!dev_workspace || ((uintptr_t)dev_workspace % kAlignB) != 0)
    return bfail(nullptr, WBLBE_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < ctl.total + kAlignB)
    return bfail(nullptr, WBLBE_ENOMEM, "workspace smaller than the control region (%zu bytes)",
                 ctl.total);
  wblbe_batch* b = new (std::nothrow) wblbe_batch();
  if (!b) return bfail(nullptr, WBLBE_ENOMEM, "host allocation failed");
  b->scheme = scheme;
  b->precision = precision;
  b->elem = precision == WBLBE_FP64 ? 8 : 4;
  b->max_cases = max_cases;
  b->max_tiles = max_tiles;
  b->max_case_nodes = max_case_nodes;
  b->cfg = *config;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return bfail(nullptr, WBLBE_ECUDA, "no CUDA device / stream");
  }
  b->ws = static_cast<unsigned char*>(dev_workspace);
  b->ws_bytes = workspace_bytes;
  b->d_cases = reinterpret_cast<CaseDev*>(b->ws + ctl.cases);
  b->d_tiles = reinterpret_cast<TileDev*>(b->ws + ctl.tiles);
  b->d_run = reinterpret_cast<RunCase*>(b->ws + ctl.run);
  b->d_done = reinterpret_cast<int*>(b->ws + ctl.done);
  b->d_head = reinterpret_cast<int*>(b->ws + ctl.head);
  b->d_status = reinterpret_cast<int*>(b->ws + ctl.status);
  b->d_desc = reinterpret_cast<BatchDesc*>(b->ws + ctl.desc);
  b->d_tile_stats = reinterpret_cast<double*>(b->ws + ctl.tile_stats);
  b->d_case_stats = reinterpret_cast<double*>(b->ws + ctl.case_stats);
  b->d_partials = reinterpret_cast<double*>(b->ws + ctl.partials);
  b->d_stage = reinterpret_cast<double*>(b->ws + ctl.stage);
  b->arena = b->ws + ctl.total;
  b->arena_bytes = (workspace_bytes - ctl.total) / kAlignB * kAlignB;
  b->free_ranges[0] = b->arena_bytes;
  b->cases.resize(max_cases);
  cudaError_t e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
  BatchDesc desc{0, config->steps_per_launch, 0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_desc, &desc, sizeof(desc), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    cudaStreamDestroy(b->capture_stream);
    delete b;
    return bfail(nullptr, WBLBE_ECUDA, "batch init: %s", cudaGetErrorString(e));
  }
  *out = b;
  return WBLBE_OK;
}

wblbe_status wblbe_batch_set_config(wblbe_batch_handle b, const wblbe_batch_config* config) {
  if (!b) return bfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (!config || (config->tile_x != 32 && config->tile_x != 64 && config->tile_x != 128 &&
                  config->tile_x != 256) ||
      config->rows_per_tile < 4 || config->steps_per_launch < 1)
    return bfail(b, WBLBE_EINVAL, "config: tile_x 32/64/128/256, rows_per_tile >= 4, steps >= 1");
  const bool retile = config->tile_x != b->cfg.tile_x || config->rows_per_tile != b->cfg.rows_per_tile;
  if (config->tile_x != b->cfg.tile_x) drop_batch_graph(b);
  b->cfg = *config;
  if (retile) b->tiles_dirty = true;
  return WBLBE_OK;
}

wblbe_status wblbe_batch_get_config(wblbe_batch_handle b, wblbe_batch_config* config) {
  if (!b || !config) return bfail(b, WBLBE_EINVAL, "NULL argument");
  *config = b->cfg;
  return WBLBE_OK;
}

wblbe_status wblbe_batch_set_wait_limit(wblbe_batch_handle b, int64_t spins) {
  if (!b) return bfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (spins < 1) return bfail(b, WBLBE_EINVAL, "spins must be >= 1");
  b->spins = spins;
  drop_batch_graph(b);
  return WBLBE_OK;
}

wblbe_status wblbe_batch_admit(wblbe_batch_handle b, const wblbe_params* params, const double* rho,
                               double umax_tol, int64_t max_steps, int64_t* case_id) {
  if (!b) return bfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  char why[256];
  if (!batch_params_valid(b, params, why, sizeof(why))) return bfail(b, WBLBE_EINVAL, "%s", why);
  if (!rho || !case_id || !(umax_tol >= 0.0) || max_steps < 0)
    return bfail(b, WBLBE_EINVAL, "need rho, case_id, umax_tol >= 0, max_steps >= 0");
  int slot = -1;
  for (int i = 0; i < b->max_cases; ++i)
    if (!b->cases[i].used) { slot = i; break; }
  if (slot < 0) return bfail(b, WBLBE_ENOMEM, "no free case slot (%d in use)", b->max_cases);
  // tiles this case adds (running cases' tile lists are cached per config)
  wblbe_batch::Case& c = b->cases[slot];
  c = wblbe_batch::Case();
  c.p = *params;
  c.id = b->next_id;
  {
    wblbe_status st = ensure_case_tiles(b, c);
    if (st != WBLBE_OK) { c = wblbe_batch::Case(); return st; }
    long long ntiles = (long long)c.tiles.size();
    for (size_t ci = 0; ci < b->cases.size(); ++ci) {
      auto& o = b->cases[ci];
      if ((int)ci == slot || !o.used || !o.running) continue;
      st = ensure_case_tiles(b, o);
      if (st != WBLBE_OK) { c = wblbe_batch::Case(); return st; }
      ntiles += (long long)o.tiles.size();
    }
    if (ntiles > b->max_tiles) {
      c = wblbe_batch::Case();
      return bfail(b, WBLBE_ENOMEM, "tile table full (%lld > %d)", ntiles, b->max_tiles);
    }
  }
  const size_t bytes = case_bytes(params, b->elem);
  size_t off = 0;
  if (!alloc_range(b, bytes, &off)) {
    c = wblbe_batch::Case();
    return bfail(b, WBLBE_ENOMEM, "arena has no free range of %zu bytes", bytes);
  }
  c.used = true;
  c.running = true;
  c.reported = false;
  c.state = WBLBE_CASE_RUNNING;
  c.p = *params;
  c.pitch = case_pitch(params->nx, b->elem);
  c.plane = (long long)c.pitch * params->ny;
  c.off = off;
  c.bytes = bytes;
  c.tol = umax_tol;
  c.max_steps = max_steps;
  b->tiles_dirty = true;                  // the tile table is rebuilt before the next launch
  const wblbe_status st = admit_device(b, slot, rho);
  if (st != WBLBE_OK) {
    // give the slot and its arena range back (the message stays in b->err)
    free_range(b, c.off, c.bytes);
    c = wblbe_batch::Case();
    return st;
  }
  b->next_id++;
  *case_id = c.id;
  return WBLBE_OK;
}

wblbe_status wblbe_batch_advance(wblbe_batch_handle b, int32_t launches) {
  if (!b) return bfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  if (launches < 1) return bfail(b, WBLBE_EINVAL, "launches must be >= 1");
  const int K = b->cfg.steps_per_launch;
  std::vector<double> cs((size_t)b->max_cases * kStatRec);
  for (int l = 0; l < launches; ++l) {
    if (b->tiles_dirty) {
      wblbe_status st = rebuild_tiles(b);
      if (st != WBLBE_OK) return st;
    }
    if (b->nrun == 0) return WBLBE_OK;
    BatchDesc desc{b->ntiles, K, b->nrun, 0};
    BCU(b, cudaMemcpyAsync(b->d_desc, &desc, sizeof(desc), cudaMemcpyHostToDevice, b->stream));
    if (!b->graph_valid) {
      wblbe_status st = build_batch_graph(b);
      if (st != WBLBE_OK) return st;
    }
    BCU(b, cudaGraphLaunch(b->graph, b->stream));
    b->launches += 2;                      // persistent + finish kernel
    int status = 0;
    BCU(b, cudaMemcpyAsync(cs.data(), b->d_case_stats, cs.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, b->stream));
    BCU(b, cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCU(b, cudaStreamSynchronize(b->stream));
    if (status != 0)
      return bfail(b, WBLBE_ETIMEOUT, "a tile wait gave up; the batch state is invalid");
    // check every running case at the launch boundary
    for (const RunCase& rc : b->run_host) {
      auto& c = b->cases[rc.c];
      c.steps += K;
      if (K & 1) c.cur ^= 1;
      const double* v = cs.data() + (size_t)rc.c * kStatRec;
      c.last.step = c.steps;
      c.last.mass = v[0];
      c.last.kinetic = v[1];
      c.last.umax = v[2];
      c.last.mu_min = v[3];
      c.last.mu_max = v[4];
      c.last.nonfinite = v[5] != 0.0 || !std::isfinite(v[0]);
      c.last.mass_drift_rel = c.mass0 != 0.0 ? (v[0] - c.mass0) / c.mass0 : 0.0;
      int state = WBLBE_CASE_RUNNING;
      if (c.last.nonfinite) state = WBLBE_CASE_UNSTABLE;
      else if (c.last.umax < c.tol) state = WBLBE_CASE_CONVERGED;
      else if (c.steps >= c.max_steps) state = WBLBE_CASE_MAXSTEPS;
      if (state != WBLBE_CASE_RUNNING) {
        c.state = state;
        c.running = false;
        b->tiles_dirty = true;
      }
    }
  }
  return WBLBE_OK;
}

wblbe_status wblbe_batch_poll(wblbe_batch_handle b, int64_t* ids, int32_t cap, int32_t* n_done) {
  if (!b || !n_done || (cap > 0 && !ids)) return bfail(b, WBLBE_EINVAL, "NULL argument");
  int n = 0;
  for (auto& c : b->cases) {
    if (n >= cap) break;
    if (c.used && !c.running && !c.reported) {
      ids[n++] = c.id;
      c.reported = true;
    }
  }
  *n_done = n;
  return WBLBE_OK;
}

wblbe_status wblbe_batch_case_info(wblbe_batch_handle b, int64_t case_id, wblbe_case_info* info) {
  if (!b || !info) return bfail(b, WBLBE_EINVAL, "NULL argument");
  const int ci = find_case(b, case_id);
  if (ci < 0) return bfail(b, WBLBE_EINVAL, "unknown case %lld", (long long)case_id);
  const auto& c = b->cases[ci];
  info->case_id = c.id;
  info->state = c.state;
  info->steps = c.steps;
  info->stats = c.last;
  return WBLBE_OK;
}

wblbe_status wblbe_batch_fetch(wblbe_batch_handle b, int64_t case_id, double* rho, double* ux,
                               double* uy, double* mu, wblbe_stats* stats) {
  if (!b) return bfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  const int ci = find_case(b, case_id);
  if (ci < 0) return bfail(b, WBLBE_EINVAL, "unknown case %lld", (long long)case_id);
  const auto& c = b->cases[ci];
  const size_t nodes = (size_t)c.p.nx * c.p.ny;
  double* outs[4] = {rho, ux, uy, mu};
  bool any = false;
  for (int k = 0; k < 4; ++k) {
    if (!outs[k]) continue;
    any = true;
    double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
    dev[k] = b->d_stage;
    wblbe_status st = case_moments(b, c, dev[0], dev[1], dev[2], dev[3], nullptr);
    if (st != WBLBE_OK) return st;
    BCU(b, cudaMemcpyAsync(outs[k], b->d_stage, nodes * sizeof(double), cudaMemcpyDeviceToHost,
                           b->stream));
  }
  if (!any) {
    wblbe_status st = case_moments(b, c, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != WBLBE_OK) return st;
  }
  double v[kStatRec];
  BCU(b, cudaMemcpyAsync(v, scratch_stats(b), sizeof(v), cudaMemcpyDeviceToHost, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  if (stats) {
    stats->step = c.steps;
    stats->mass = v[0];
    stats->kinetic = v[1];
    stats->umax = v[2];
    stats->mu_min = v[3];
    stats->mu_max = v[4];
    stats->nonfinite = v[5] != 0.0 || !std::isfinite(v[0]);
    stats->mass_drift_rel = c.mass0 != 0.0 ? (v[0] - c.mass0) / c.mass0 : 0.0;
  }
  return WBLBE_OK;
}

wblbe_status wblbe_batch_get_populations(wblbe_batch_handle b, int64_t case_id, double* f) {
  if (!b || !f) return bfail(b, WBLBE_EINVAL, "NULL argument");
  const int ci = find_case(b, case_id);
  if (ci < 0) return bfail(b, WBLBE_EINVAL, "unknown case %lld", (long long)case_id);
  const auto& c = b->cases[ci];
  const size_t nodes = (size_t)c.p.nx * c.p.ny;
  LayoutParams lp = case_layout(c);
  dim3 grid((c.p.nx + 127) / 128, c.p.ny);
  const unsigned char* pops = b->arena + c.off + (c.cur ? c.bytes / 2 : 0);
  for (int i = 0; i < 9; ++i) {
    if (b->precision == WBLBE_FP64)
      batch_get_pops_kernel<double><<<grid, 128, 0, b->stream>>>(
          reinterpret_cast<const double*>(pops), b->d_stage, c.p.nx, c.p.ny, c.pitch, c.plane, lp, i);
    else
      batch_get_pops_kernel<float><<<grid, 128, 0, b->stream>>>(
          reinterpret_cast<const float*>(pops), b->d_stage, c.p.nx, c.p.ny, c.pitch, c.plane, lp, i);
    BCU(b, cudaGetLastError());
    BCU(b, cudaMemcpyAsync(f + i * nodes, b->d_stage, nodes * sizeof(double),
                           cudaMemcpyDeviceToHost, b->stream));
  }
  BCU(b, cudaStreamSynchronize(b->stream));
  return WBLBE_OK;
}

wblbe_status wblbe_batch_retire(wblbe_batch_handle b, int64_t case_id) {
  if (!b) return bfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  const int ci = find_case(b, case_id);
  if (ci < 0) return bfail(b, WBLBE_EINVAL, "unknown case %lld", (long long)case_id);
  BCU(b, cudaStreamSynchronize(b->stream));
  auto& c = b->cases[ci];
  const bool was_running = c.running;
  free_range(b, c.off, c.bytes);
  c = wblbe_batch::Case();
  if (was_running) b->tiles_dirty = true;
  return WBLBE_OK;
}

wblbe_status wblbe_batch_counts(wblbe_batch_handle b, int32_t* resident, int32_t* running,
                                int32_t* tiles, size_t* arena_free) {
  if (!b) return bfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  int res = 0, run = 0, nt = 0;
  for (auto& c : b->cases) {
    if (!c.used) continue;
    ++res;
    if (c.running) {
      ++run;
      if (ensure_case_tiles(b, c) == WBLBE_OK) nt += (int)c.tiles.size();
    }
  }
  size_t fr = 0;
  for (const auto& r : b->free_ranges) fr += r.second;
  if (resident) *resident = res;
  if (running) *running = run;
  if (tiles) *tiles = nt;
  if (arena_free) *arena_free = fr;
  return WBLBE_OK;
}

int64_t wblbe_batch_kernel_launches(wblbe_batch_handle b) { return b ? b->launches : -1; }

wblbe_status wblbe_batch_destroy(wblbe_batch_handle b) {
  if (!b) return bfail(nullptr, WBLBE_EINVAL, "handle is NULL");
  cudaStreamSynchronize(b->stream);
  drop_batch_graph(b);
  cudaStreamDestroy(b->capture_stream);
  delete b;
  return WBLBE_OK;
}

const char* wblbe_batch_last_error(wblbe_batch_handle b) { return b ? b->err : g_batch_error; }

}  // extern "C"

namespace wblbe {
// bounds-check count of this translation unit's kernels (see lbm_kernels.cuh)
unsigned int batch_bounds_errors(bool reset) { return read_bounds_errors(reset); }
}  // namespace wblbe
