// float32 instantiations of the marching sweeps (mixed-precision V-cycle:
// finest level with bfloat16 moduli, coarse levels with float32 element
// matrices).  These kernels are bound by instruction issue and memory
// latency, so they use two node columns per lane and load several rows ahead
// of the arithmetic.
#include "mto_launch.h"

namespace mto {

// Rows of lookahead per source and mode, bounded by the registers one row of
// loads takes.
template <int SRC, int MODE, bool DOT> constexpr int lookahead() {
  if (SRC == SRC_CMOM && MODE == MODE_PSMOOTH) return 1;
  if (SRC == SRC_FINEBF && MODE == MODE_SMOOTH0 && DOT) return 1;  // float64 r and q per row
  if (DOT || MODE == MODE_PSMOOTH || SRC == SRC_CFINE || SRC == SRC_CMOM) return 2;
  return 3;
}

template <int SRC, int MODE, bool DOT>
static cudaError_t go(SweepParams<float> p, int tw, int num_sms, cudaStream_t s) {
  constexpr int COLS = sweep_cols_of(false, SRC, MODE);
  constexpr int PF = lookahead<SRC, MODE, DOT>();
  void (*kernel)(SweepParams<float>);
  if constexpr (MODE == MODE_POST2) kernel = post2_kernel<SRC, 2>;
  else if constexpr (MODE == MODE_PRE2) kernel = pre2_kernel<SRC, 2>;
  else if constexpr (COLS == 2) kernel = sweep2_kernel<float, SRC, MODE, DOT, float2, PF>;
  else kernel = sweep_kernel<float, SRC, MODE, DOT, float2, PF>;
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
cudaError_t launch_sweep<float>(int src, int mode, bool dot, bool zfloat, SweepParams<float> p,
                                int tw, int num_sms, cudaStream_t s) {
  (void)zfloat;
  if (src == SRC_FINEBF) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_FINEBF, MODE_APPLY, false>(p, tw, num_sms, s);
      case MODE_SMOOTH:
        return dot ? go<SRC_FINEBF, MODE_SMOOTH, true>(p, tw, num_sms, s)
                   : go<SRC_FINEBF, MODE_SMOOTH, false>(p, tw, num_sms, s);
      case MODE_SMOOTH0:  // with dot: carrying the CG update
        return dot ? go<SRC_FINEBF, MODE_SMOOTH0, true>(p, tw, num_sms, s)
                   : go<SRC_FINEBF, MODE_SMOOTH0, false>(p, tw, num_sms, s);
      case MODE_PSMOOTH:
        return dot ? go<SRC_FINEBF, MODE_PSMOOTH, true>(p, tw, num_sms, s)
                   : go<SRC_FINEBF, MODE_PSMOOTH, false>(p, tw, num_sms, s);
      case MODE_RESTRICT: return go<SRC_FINEBF, MODE_RESTRICT, false>(p, tw, num_sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (src == SRC_CFINE) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_CFINE, MODE_APPLY, false>(p, tw, num_sms, s);
      case MODE_SMOOTH: return go<SRC_CFINE, MODE_SMOOTH, false>(p, tw, num_sms, s);
      case MODE_SMOOTH0: return go<SRC_CFINE, MODE_SMOOTH0, false>(p, tw, num_sms, s);
      case MODE_PSMOOTH: return go<SRC_CFINE, MODE_PSMOOTH, false>(p, tw, num_sms, s);
      case MODE_RESTRICT: return go<SRC_CFINE, MODE_RESTRICT, false>(p, tw, num_sms, s);
      case MODE_POST2: return go<SRC_CFINE, MODE_POST2, false>(p, tw, num_sms, s);
      case MODE_PRE2: return go<SRC_CFINE, MODE_PRE2, false>(p, tw, num_sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (src == SRC_CMOM) {
    switch (mode) {
      case MODE_APPLY: return go<SRC_CMOM, MODE_APPLY, false>(p, tw, num_sms, s);
      case MODE_SMOOTH: return go<SRC_CMOM, MODE_SMOOTH, false>(p, tw, num_sms, s);
      case MODE_SMOOTH0: return go<SRC_CMOM, MODE_SMOOTH0, false>(p, tw, num_sms, s);
      case MODE_PSMOOTH: return go<SRC_CMOM, MODE_PSMOOTH, false>(p, tw, num_sms, s);
      case MODE_RESTRICT: return go<SRC_CMOM, MODE_RESTRICT, false>(p, tw, num_sms, s);
      case MODE_POST2: return go<SRC_CMOM, MODE_POST2, false>(p, tw, num_sms, s);
      case MODE_PRE2: return go<SRC_CMOM, MODE_PRE2, false>(p, tw, num_sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mto
