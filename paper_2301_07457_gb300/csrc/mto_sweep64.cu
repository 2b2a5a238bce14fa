// float64 instantiations of the marching sweeps (finest level with float64
// moduli, coarse levels with float64 element matrices), and the launch-shape
// rule shared by all sweeps.  The float64 kernels are bound by the FP64 pipe,
// so one step of load lookahead suffices.
#include "mto_launch.h"

namespace mto {

SweepShape sweep_shape(const Grid& g, int mode, int target_warps, int cols) {
  SweepShape sh;
  if (mode == MODE_PRE2) {
    // 29 output coarse columns per warp, coarse rows per task as for the
    // restriction sweep.
    const int nxc = g.nx / 2, nyc = g.ny / 2;
    sh.nstrips = (nxc + 1 + PRE2_CSTRIDE - 1) / PRE2_CSTRIDE;
    const int want = target_warps / sh.nstrips > 1 ? target_warps / sh.nstrips : 1;
    int hc = (nyc + 1 + want - 1) / want;
    hc = hc < 1 ? 1 : (hc > 32 ? 32 : hc);
    sh.H = 2 * hc;
    sh.nchunks = (nyc + 1 + hc - 1) / hc;
  } else if (mode == MODE_POST2) {
    // 60 output columns per warp, rows as for a smoothing sweep.
    sh.nstrips = (g.nx + 1 + POST2_STRIDE - 1) / POST2_STRIDE;
    const int want = target_warps / sh.nstrips > 1 ? target_warps / sh.nstrips : 1;
    int h = (g.ny + 1 + want - 1) / want;
    h = h < 1 ? 1 : (h > 64 ? 64 : h);
    sh.H = h;
    sh.nchunks = (g.ny + 1 + h - 1) / h;
  } else if (mode == MODE_RESTRICT) {
    // Coarse columns per warp: 14 (one column per lane) or 30 (two).
    const int cstride = cols == 2 ? SWEEP2_RSTRIDE / 2 : SWEEP_RSTRIDE / 2;
    const int nxc = g.nx / 2, nyc = g.ny / 2;
    sh.nstrips = (nxc + 1 + cstride - 1) / cstride;
    const int want = target_warps / sh.nstrips > 1 ? target_warps / sh.nstrips : 1;
    int hc = (nyc + 1 + want - 1) / want;
    hc = hc < 1 ? 1 : (hc > 32 ? 32 : hc);
    sh.H = 2 * hc;
    sh.nchunks = (nyc + 1 + hc - 1) / hc;
  } else {
    // Output node columns per warp: 30 ([30 s, 30 s + 29]) or 62 ([62 s - 1, 62 s + 60]).
    sh.nstrips = cols == 2 ? (g.nx + 2 + SWEEP2_STRIDE - 1) / SWEEP2_STRIDE
                           : (g.nx + 1 + SWEEP_STRIDE - 1) / SWEEP_STRIDE;
    const int want = target_warps / sh.nstrips > 1 ? target_warps / sh.nstrips : 1;
    // One row per task on small levels: with the halo step, two steps whose
    // loads all fit the lookahead ring, so the sweep costs one memory round
    // trip instead of two.
    int h = (g.ny + 1 + want - 1) / want;
    h = h < 1 ? 1 : (h > 64 ? 64 : h);
    sh.H = h;
    sh.nchunks = (g.ny + 1 + h - 1) / h;
  }
  const long long warps = (long long)sh.nstrips * sh.nchunks;
  sh.nblocks = (int)((warps + SWEEP_NT / 32 - 1) / (SWEEP_NT / 32));
  return sh;
}

int sweep_cols(bool f64, int src, int mode) { return sweep_cols_of(f64, src, mode); }

template <int SRC, int MODE, bool DOT, typename ZT>
static cudaError_t go(SweepParams<double> p, int tw, int num_sms, cudaStream_t s) {
  constexpr int COLS = sweep_cols_of(true, SRC, MODE);
  void (*kernel)(SweepParams<double>);
  if constexpr (COLS == 2) kernel = sweep2_kernel<double, SRC, MODE, DOT, ZT, 1>;
  else kernel = sweep_kernel<double, SRC, MODE, DOT, ZT, 1>;
  if (tw <= 0) {
    static const int wave = full_wave_warps(kernel, num_sms);  // same for every device of a run
    tw = wave;
  }
  const SweepShape sh = sweep_shape(p.g, MODE, tw, COLS);
  p.nstrips = sh.nstrips;
  p.nchunks = sh.nchunks;
  p.H = sh.H;
  return launch_pdl(kernel, sh.nblocks, SWEEP_NT, 0, s, p);
}

template <>
cudaError_t launch_sweep<double>(int src, int mode, bool dot, bool zfloat, SweepParams<double> p,
                                 int tw, int num_sms, cudaStream_t s) {
  if (src == SRC_FINE64) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_FINE64, MODE_APPLY, false, double2>(p, tw, num_sms, s);
      case MODE_RESID: return go<SRC_FINE64, MODE_RESID, false, double2>(p, tw, num_sms, s);
      case MODE_KP:
        return zfloat ? go<SRC_FINE64, MODE_KP, false, float2>(p, tw, num_sms, s)
                      : go<SRC_FINE64, MODE_KP, false, double2>(p, tw, num_sms, s);
      case MODE_SMOOTH:
        return dot ? go<SRC_FINE64, MODE_SMOOTH, true, double2>(p, tw, num_sms, s)
                   : go<SRC_FINE64, MODE_SMOOTH, false, double2>(p, tw, num_sms, s);
      case MODE_SMOOTH0: return go<SRC_FINE64, MODE_SMOOTH0, false, double2>(p, tw, num_sms, s);
      case MODE_PSMOOTH:
        return dot ? go<SRC_FINE64, MODE_PSMOOTH, true, double2>(p, tw, num_sms, s)
                   : go<SRC_FINE64, MODE_PSMOOTH, false, double2>(p, tw, num_sms, s);
      case MODE_RESTRICT: return go<SRC_FINE64, MODE_RESTRICT, false, double2>(p, tw, num_sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (src == SRC_COARSE) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_COARSE, MODE_APPLY, false, double2>(p, tw, num_sms, s);
      case MODE_SMOOTH: return go<SRC_COARSE, MODE_SMOOTH, false, double2>(p, tw, num_sms, s);
      case MODE_SMOOTH0: return go<SRC_COARSE, MODE_SMOOTH0, false, double2>(p, tw, num_sms, s);
      case MODE_PSMOOTH: return go<SRC_COARSE, MODE_PSMOOTH, false, double2>(p, tw, num_sms, s);
      case MODE_RESTRICT: return go<SRC_COARSE, MODE_RESTRICT, false, double2>(p, tw, num_sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mto
