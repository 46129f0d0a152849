// Strip-kernel instantiations of the two variants of the standard LBE that
// Sec. II of Guo, arXiv 2012.11075 compares with: the pressure-form
// interaction force (scheme code 2) and the forcing term of Guo's textbook
// (scheme code 3).  The single-lattice runtime (wblbe.cu) dispatches to them.
#include "strip_launch.cuh"

namespace wblbe {

cudaError_t launch_variant(int sch, bool fp64, bool moments, const void* src, void* dst,
                           const KParams& kp, const MomentsOut& mo, int tile, cudaStream_t s) {
  if (sch == kSchPressure)
    return launch_scheme<kSchPressure>(fp64, moments, src, dst, kp, mo, tile, s);
  if (sch == kSchTextbook)
    return launch_scheme<kSchTextbook>(fp64, moments, src, dst, kp, mo, tile, s);
  return cudaErrorInvalidValue;
}

int resident_variant(int sch, bool fp64, int tile) {
  return sch == kSchPressure ? resident_scheme<kSchPressure>(fp64, tile)
                             : resident_scheme<kSchTextbook>(fp64, tile);
}

cudaError_t allow_smem_variants() {
  cudaError_t e = cudaSuccess, r;
  if ((r = allow_smem_scheme<kSchPressure>()) != cudaSuccess) e = r;
  if ((r = allow_smem_scheme<kSchTextbook>()) != cudaSuccess) e = r;
  return e;
}

}  // namespace wblbe
