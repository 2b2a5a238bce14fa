// float64 instantiations of the marching sweeps (finest level with float64
// moduli, coarse levels with float64 element matrices).  These kernels are
// bound by the FP64 pipe, so one step of load lookahead suffices.
#include "mto_launch.h"

namespace mto {

SweepShape sweep_shape(const Grid& g, int mode, int target_warps) {
  SweepShape sh;
  if (mode == MODE_RESTRICT) {
    const int nxc = g.nx / 2, nyc = g.ny / 2;
    sh.nstrips = (nxc + 1 + SWEEP_RSTRIDE / 2 - 1) / (SWEEP_RSTRIDE / 2);
    const int want = target_warps / sh.nstrips > 1 ? target_warps / sh.nstrips : 1;
    int hc = (nyc + 1 + want - 1) / want;
    hc = hc < 1 ? 1 : (hc > 32 ? 32 : hc);
    sh.H = 2 * hc;
    sh.nchunks = (nyc + 1 + hc - 1) / hc;
  } else {
    sh.nstrips = (g.nx + 1 + SWEEP_STRIDE - 1) / SWEEP_STRIDE;
    const int want = target_warps / sh.nstrips > 1 ? target_warps / sh.nstrips : 1;
    int h = (g.ny + 1 + want - 1) / want;
    h = h < 2 ? 2 : (h > 64 ? 64 : h);
    sh.H = h;
    sh.nchunks = (g.ny + 1 + h - 1) / h;
  }
  const long long warps = (long long)sh.nstrips * sh.nchunks;
  sh.nblocks = (int)((warps + SWEEP_NT / 32 - 1) / (SWEEP_NT / 32));
  return sh;
}

template <int SRC, int MODE, bool DOT, typename ZT>
static cudaError_t go(const SweepParams<double>& p, const SweepShape& sh, cudaStream_t s) {
  sweep_kernel<double, SRC, MODE, DOT, ZT, 1><<<sh.nblocks, SWEEP_NT, 0, s>>>(p);
  return cudaGetLastError();
}

template <>
cudaError_t launch_sweep<double>(int src, int mode, bool dot, bool zfloat, SweepParams<double> p,
                                 const SweepShape& sh, cudaStream_t s) {
  p.nstrips = sh.nstrips;
  p.nchunks = sh.nchunks;
  p.H = sh.H;
  if (src == SRC_FINE64) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_FINE64, MODE_APPLY, false, double2>(p, sh, s);
      case MODE_RESID: return go<SRC_FINE64, MODE_RESID, false, double2>(p, sh, s);
      case MODE_KP:
        return zfloat ? go<SRC_FINE64, MODE_KP, false, float2>(p, sh, s)
                      : go<SRC_FINE64, MODE_KP, false, double2>(p, sh, s);
      case MODE_SMOOTH:
        return dot ? go<SRC_FINE64, MODE_SMOOTH, true, double2>(p, sh, s)
                   : go<SRC_FINE64, MODE_SMOOTH, false, double2>(p, sh, s);
      case MODE_SMOOTH0: return go<SRC_FINE64, MODE_SMOOTH0, false, double2>(p, sh, s);
      case MODE_PSMOOTH:
        return dot ? go<SRC_FINE64, MODE_PSMOOTH, true, double2>(p, sh, s)
                   : go<SRC_FINE64, MODE_PSMOOTH, false, double2>(p, sh, s);
      case MODE_RESTRICT: return go<SRC_FINE64, MODE_RESTRICT, false, double2>(p, sh, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (src == SRC_COARSE) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_COARSE, MODE_APPLY, false, double2>(p, sh, s);
      case MODE_SMOOTH: return go<SRC_COARSE, MODE_SMOOTH, false, double2>(p, sh, s);
      case MODE_SMOOTH0: return go<SRC_COARSE, MODE_SMOOTH0, false, double2>(p, sh, s);
      case MODE_PSMOOTH: return go<SRC_COARSE, MODE_PSMOOTH, false, double2>(p, sh, s);
      case MODE_RESTRICT: return go<SRC_COARSE, MODE_RESTRICT, false, double2>(p, sh, s);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mto
