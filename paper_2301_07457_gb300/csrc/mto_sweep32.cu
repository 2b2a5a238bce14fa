// float32 instantiations of the marching sweeps (mixed-precision V-cycle:
// finest level with bfloat16 moduli, coarse levels with float32 element
// matrices).  These kernels are bound by memory, so loads run several steps
// ahead of the arithmetic.
#include "mto_launch.h"

namespace mto {

template <int SRC, int MODE, bool DOT, int PF>
static cudaError_t go(const SweepParams<float>& p, const SweepShape& sh, cudaStream_t s) {
  sweep_kernel<float, SRC, MODE, DOT, float2, PF><<<sh.nblocks, SWEEP_NT, 0, s>>>(p);
  return cudaGetLastError();
}

template <>
cudaError_t launch_sweep<float>(int src, int mode, bool dot, bool zfloat, SweepParams<float> p,
                                const SweepShape& sh, cudaStream_t s) {
  (void)zfloat;
  p.nstrips = sh.nstrips;
  p.nchunks = sh.nchunks;
  p.H = sh.H;
  if (src == SRC_FINEBF) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_FINEBF, MODE_APPLY, false, 3>(p, sh, s);
      case MODE_SMOOTH:
        return dot ? go<SRC_FINEBF, MODE_SMOOTH, true, 3>(p, sh, s)
                   : go<SRC_FINEBF, MODE_SMOOTH, false, 3>(p, sh, s);
      case MODE_PSMOOTH:
        return dot ? go<SRC_FINEBF, MODE_PSMOOTH, true, 2>(p, sh, s)
                   : go<SRC_FINEBF, MODE_PSMOOTH, false, 2>(p, sh, s);
      case MODE_RESTRICT: return go<SRC_FINEBF, MODE_RESTRICT, false, 3>(p, sh, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (src == SRC_CFINE) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_CFINE, MODE_APPLY, false, 2>(p, sh, s);
      case MODE_SMOOTH: return go<SRC_CFINE, MODE_SMOOTH, false, 3>(p, sh, s);
      case MODE_SMOOTH0: return go<SRC_CFINE, MODE_SMOOTH0, false, 3>(p, sh, s);
      case MODE_PSMOOTH: return go<SRC_CFINE, MODE_PSMOOTH, false, 2>(p, sh, s);
      case MODE_RESTRICT: return go<SRC_CFINE, MODE_RESTRICT, false, 3>(p, sh, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (src == SRC_COARSE) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_COARSE, MODE_APPLY, false, 2>(p, sh, s);
      case MODE_SMOOTH: return go<SRC_COARSE, MODE_SMOOTH, false, 2>(p, sh, s);
      case MODE_SMOOTH0: return go<SRC_COARSE, MODE_SMOOTH0, false, 2>(p, sh, s);
      case MODE_PSMOOTH: return go<SRC_COARSE, MODE_PSMOOTH, false, 2>(p, sh, s);
      case MODE_RESTRICT: return go<SRC_COARSE, MODE_RESTRICT, false, 2>(p, sh, s);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mto
