// float32 instantiations of the marching sweeps (mixed-precision V-cycle:
// finest level with bfloat16 moduli, coarse levels with float32 element
// matrices).  These kernels are bound by instruction issue and memory
// latency, so they use two node columns per lane and load several rows ahead
// of the arithmetic.
#include "mto_launch.h"

namespace mto {

// Rows of lookahead per source and mode: bounded by the registers one row of
// loads takes (a coarse element pair is 26 floats).
template <int SRC, int MODE, bool DOT> constexpr int lookahead() {
  if (SRC == SRC_COARSE) return 2;
  if (DOT || MODE == MODE_PSMOOTH || SRC == SRC_CFINE) return 2;
  return 3;
}

template <int SRC, int MODE, bool DOT>
static cudaError_t go(SweepParams<float> p, int tw, cudaStream_t s) {
  constexpr int COLS = sweep_cols_of(false, SRC, MODE);
  constexpr int PF = lookahead<SRC, MODE, DOT>();
  const SweepShape sh = sweep_shape(p.g, MODE, tw, COLS);
  p.nstrips = sh.nstrips;
  p.nchunks = sh.nchunks;
  p.H = sh.H;
  if constexpr (COLS == 2) {
    return launch_pdl(sweep2_kernel<float, SRC, MODE, DOT, float2, PF>, sh.nblocks, SWEEP_NT, 0, s, p);
  } else {
    return launch_pdl(sweep_kernel<float, SRC, MODE, DOT, float2, PF>, sh.nblocks, SWEEP_NT, 0, s, p);
  }
}

template <>
cudaError_t launch_sweep<float>(int src, int mode, bool dot, bool zfloat, SweepParams<float> p,
                                int tw, cudaStream_t s) {
  (void)zfloat;
  if (src == SRC_FINEBF) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_FINEBF, MODE_APPLY, false>(p, tw, s);
      case MODE_SMOOTH:
        return dot ? go<SRC_FINEBF, MODE_SMOOTH, true>(p, tw, s)
                   : go<SRC_FINEBF, MODE_SMOOTH, false>(p, tw, s);
      case MODE_SMOOTH0: return go<SRC_FINEBF, MODE_SMOOTH0, false>(p, tw, s);
      case MODE_PSMOOTH:
        return dot ? go<SRC_FINEBF, MODE_PSMOOTH, true>(p, tw, s)
                   : go<SRC_FINEBF, MODE_PSMOOTH, false>(p, tw, s);
      case MODE_RESTRICT: return go<SRC_FINEBF, MODE_RESTRICT, false>(p, tw, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (src == SRC_CFINE) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_CFINE, MODE_APPLY, false>(p, tw, s);
      case MODE_SMOOTH: return go<SRC_CFINE, MODE_SMOOTH, false>(p, tw, s);
      case MODE_SMOOTH0: return go<SRC_CFINE, MODE_SMOOTH0, false>(p, tw, s);
      case MODE_PSMOOTH: return go<SRC_CFINE, MODE_PSMOOTH, false>(p, tw, s);
      case MODE_RESTRICT: return go<SRC_CFINE, MODE_RESTRICT, false>(p, tw, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (src == SRC_COARSE) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_COARSE, MODE_APPLY, false>(p, tw, s);
      case MODE_SMOOTH: return go<SRC_COARSE, MODE_SMOOTH, false>(p, tw, s);
      case MODE_SMOOTH0: return go<SRC_COARSE, MODE_SMOOTH0, false>(p, tw, s);
      case MODE_PSMOOTH: return go<SRC_COARSE, MODE_PSMOOTH, false>(p, tw, s);
      case MODE_RESTRICT: return go<SRC_COARSE, MODE_RESTRICT, false>(p, tw, s);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mto
