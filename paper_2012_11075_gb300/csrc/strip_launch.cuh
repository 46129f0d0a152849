// Host-side launch helpers of the single-lattice strip kernel, templated on
// the scheme id.  wblbe.cu instantiates them for the standard and the
// well-balanced scheme, strip_variants.cu for the two comparison variants of
// the standard scheme (kept in a translation unit of their own so that the
// units compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

namespace wblbe {

template <typename T>
inline size_t strip_smem(int tile) {
  return strip_smem_bytes(tile, Staging<T>::kStages, sizeof(T));
}

// Allow every instantiation the dynamic shared memory it launches with.
template <typename T, int SCH, int MODE, int TX>
cudaError_t allow_smem_tx() {
  return cudaFuncSetAttribute(lbm_strip_kernel<T, SCH, MODE, TX>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)strip_smem<T>(TX));
}
template <typename T, int SCH, int MOM>
cudaError_t allow_smem_mom() {
  cudaError_t e = cudaSuccess, r;
  if ((r = allow_smem_tx<T, SCH, MOM, 32>()) != cudaSuccess) e = r;
  if ((r = allow_smem_tx<T, SCH, MOM, 64>()) != cudaSuccess) e = r;
  if ((r = allow_smem_tx<T, SCH, MOM, 128>()) != cudaSuccess) e = r;
  if ((r = allow_smem_tx<T, SCH, MOM, 256>()) != cudaSuccess) e = r;
  return e;
}
template <int SCH>
cudaError_t allow_smem_scheme() {
  cudaError_t e = cudaSuccess, r;
  if ((r = allow_smem_mom<double, SCH, kModeStep>()) != cudaSuccess) e = r;
  if ((r = allow_smem_mom<double, SCH, kModeMoments>()) != cudaSuccess) e = r;
  if ((r = allow_smem_mom<double, SCH, kModeStepStats>()) != cudaSuccess) e = r;
  if ((r = allow_smem_mom<float, SCH, kModeStep>()) != cudaSuccess) e = r;
  if ((r = allow_smem_mom<float, SCH, kModeMoments>()) != cudaSuccess) e = r;
  if ((r = allow_smem_mom<float, SCH, kModeStepStats>()) != cudaSuccess) e = r;
  return e;
}

template <typename T, int SCH, int MOM, int TX>
cudaError_t launch_tx(const void* src, void* dst, const KParams& kp, const MomentsOut& mo,
                      cudaStream_t s) {
  dim3 grid((kp.nx + TX - 1) / TX, (kp.row_hi - kp.row_lo + kp.rows - 1) / kp.rows);
  lbm_strip_kernel<T, SCH, MOM, TX><<<grid, TX, strip_smem<T>(TX), s>>>(
      static_cast<const T*>(src), static_cast<T*>(dst), kp, mo);
  return cudaGetLastError();
}

template <typename T, int SCH, int MOM>
cudaError_t launch_strip(const void* src, void* dst, const KParams& kp, const MomentsOut& mo,
                         int tile, cudaStream_t s) {
  switch (tile) {
    case 32: return launch_tx<T, SCH, MOM, 32>(src, dst, kp, mo, s);
    case 64: return launch_tx<T, SCH, MOM, 64>(src, dst, kp, mo, s);
    case 128: return launch_tx<T, SCH, MOM, 128>(src, dst, kp, mo, s);
    case 256: return launch_tx<T, SCH, MOM, 256>(src, dst, kp, mo, s);
    default: return cudaErrorInvalidValue;
  }
}

// mode: a StripMode (step, moments, step with statistics)
template <typename T, int SCH>
cudaError_t launch_mode(int mode, const void* src, void* dst, const KParams& kp,
                        const MomentsOut& mo, int tile, cudaStream_t s) {
  switch (mode) {
    case kModeStep: return launch_strip<T, SCH, kModeStep>(src, dst, kp, mo, tile, s);
    case kModeMoments: return launch_strip<T, SCH, kModeMoments>(src, dst, kp, mo, tile, s);
    case kModeStepStats: return launch_strip<T, SCH, kModeStepStats>(src, dst, kp, mo, tile, s);
    default: return cudaErrorInvalidValue;
  }
}
template <int SCH>
cudaError_t launch_scheme(bool fp64, int mode, const void* src, void* dst,
                          const KParams& kp, const MomentsOut& mo, int tile, cudaStream_t s) {
  return fp64 ? launch_mode<double, SCH>(mode, src, dst, kp, mo, tile, s)
              : launch_mode<float, SCH>(mode, src, dst, kp, mo, tile, s);
}

// Resident CTAs per SM of the step kernel at this tile width.
template <typename T, int SCH, int TX>
int resident_tx() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lbm_strip_kernel<T, SCH, kModeStep, TX>, TX,
                                                    strip_smem<T>(TX)) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}
template <typename T, int SCH>
int resident_per_sm(int tile) {
  switch (tile) {
    case 32: return resident_tx<T, SCH, 32>();
    case 64: return resident_tx<T, SCH, 64>();
    case 128: return resident_tx<T, SCH, 128>();
    default: return resident_tx<T, SCH, 256>();
  }
}
template <int SCH>
int resident_scheme(bool fp64, int tile) {
  return fp64 ? resident_per_sm<double, SCH>(tile) : resident_per_sm<float, SCH>(tile);
}

// The comparison variants (scheme codes 2 and 3), defined in strip_variants.cu.
cudaError_t launch_variant(int sch, bool fp64, int mode, const void* src, void* dst,
                           const KParams& kp, const MomentsOut& mo, int tile, cudaStream_t s);
int resident_variant(int sch, bool fp64, int tile);
cudaError_t allow_smem_variants();
// Scheme code 4 (FP64 tile kernel, 32 x 16 nodes per CTA): launch, and the
// number of per-CTA statistics records its moments pass writes.
constexpr int kSchE6 = 4;
cudaError_t launch_e6(int mode, const void* src, void* dst, const KParams& kp,
                      const MomentsOut& mo, cudaStream_t s);
int e6_partials(int nx, int ny);
// Strip-kernel launches for scheme codes 0-3 without instantiating the
// kernel templates again (defined in wblbe.cu; used by slabs.cu).
cudaError_t launch_strip_any(int sch, bool fp64, int mode, const void* src, void* dst,
                             const KParams& kp, const MomentsOut& mo, int tile, cudaStream_t s);
int resident_strip_any(int sch, bool fp64, int tile);
cudaError_t allow_smem_strip_all();
// Bounds-check counts of the other translation units (bounds-checked build).
unsigned int variants_bounds_errors(bool reset);
unsigned int batch_bounds_errors(bool reset);

}  // namespace wblbe
