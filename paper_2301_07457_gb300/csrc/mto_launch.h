// Host-side launchers of libmto's kernels (one translation unit each for the
// float64 sweeps, the float32 sweeps, the setup and the vector kernels).
#pragma once

#include <utility>

#include "mto_fused.cuh"
#include "mto_gemv.cuh"
#include "mto_sweep2.cuh"

namespace mto {

// Programmatic dependent launch for the launches of this thread (on by
// default).  Batched graphs turn it off while they capture: there, a kernel
// whose blocks wait early on SM slots would hold them from the other
// problems' concurrent branches.
extern thread_local bool g_pdl;

// Launch a kernel that calls pdl_wait() first, allowing programmatic
// dependent launch after the previous kernel on the stream (captured into
// graphs as a programmatic edge) while g_pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = g_pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Launch shape of a sweep over grid g (see mto_sweep.cuh and mto_sweep2.cuh).
// target_warps is the number of warps the launch should expose (a multiple of
// the SM count); cols is the number of node columns per lane (1 or 2).
struct SweepShape {
  int nstrips, nchunks, H, nblocks;
};
SweepShape sweep_shape(const Grid& g, int mode, int target_warps, int cols);

// Node columns per lane of the instantiation that launch_sweep uses for a
// float64 (f64) or float32 sweep of source src in mode `mode`.  Two for every
// float32 sweep (issue- and latency-bound) and for the float64 outer
// operator sweeps (K p, residuals: 3% less halo work on the FP64 pipe); one
// for the float64 V-cycle, where a pair of elements (13 float64 coefficients
// each on coarse levels) needs too many registers.
constexpr int sweep_cols_of(bool f64, int src, int mode) {
  if (f64) {
    return (src == SRC_FINE64 && (mode == MODE_KP || mode == MODE_RESID || mode == MODE_APPLY)) ? 2 : 1;
  }
  return 2;
}
int sweep_cols(bool f64, int src, int mode);

// Launch one sweep over p.g; the launch shape follows from target_warps
// (0: one full wave of the kernel on num_sms SMs).
template <typename T>
cudaError_t launch_sweep(int src, int mode, bool dot, bool zfloat, SweepParams<T> p,
                         int target_warps, int num_sms, cudaStream_t s);

// Warps of one full wave of a sweep kernel: resident blocks per SM (from its
// registers) times the SM count.
template <typename K> int full_wave_warps(K kernel, int num_sms) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, SWEEP_NT, 0) != cudaSuccess ||
      blocks < 1) {
    cudaGetLastError();
    blocks = 1;
  }
  return blocks * (SWEEP_NT / 32) * num_sms;
}

// ---- pointwise kernels (mto_vec.cu) ----
constexpr int VEC_NT = 256;
int vec_blocks(long long n, int num_sms);

// z = invd1 (.) r on the float64 finest level.
cudaError_t launch_jacobi0_fine64(const Grid& g, const double* invd1, const double2* r, double2* z,
                                  DevScalars* sc, int nblocks, cudaStream_t s);
// z = w / (KE_00 sum E) (.) r32 on the float32 finest level.
cudaError_t launch_jacobi0_finebf(const Grid& g, const __nv_bfloat16* E, float wdiag,
                                  const float2* r32, float2* z, DevScalars* sc, int nblocks,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_jacobi0_coarse(const Grid& g, const typename V2<T>::t* invd2,
                                  const typename V2<T>::t* b, typename V2<T>::t* z,
                                  DevScalars* sc, int nblocks, cudaStream_t s);
// x += alpha p; r -= alpha q; rr = |r|^2 (FIN_UPDATE).
// r -= alpha q, rr = |r|^2 (FIN_UPDATE: the x step becomes pending); r32 =
// float(r) when not null.
cudaError_t launch_update(const Grid& g, double2* r, float2* r32, const double2* q,
                          double* partials, unsigned* ticket, DevScalars* sc, int nblocks,
                          cudaStream_t s);
// x += alpha p[p_par] when the x step is pending (after the PCG loop).
cudaError_t launch_x_step(const Grid& g, double2* x, const double2* p0, const double2* p1,
                          const DevScalars* sc, int nblocks, cudaStream_t s);
// sum a.b over n double2 values (finish kind applied to sc, result also to out_value).
cudaError_t launch_dot(long long n, const double2* a, const double2* b, double* partials,
                       unsigned* ticket, DevScalars* sc, int finish, double* out_value,
                       int nblocks, cudaStream_t s);
// dense [ny+1][nx+1][2] <-> padded layout (pack zeroes clamped DOFs).
// With nonzero != NULL, sets *nonzero = 1 when any packed value is non-zero.
cudaError_t launch_pack(const Grid& g, const double* src, double2* dst, cudaStream_t s, int num_sms,
                        int* nonzero = nullptr);
cudaError_t launch_unpack(const Grid& g, const double2* src, double* dst, cudaStream_t s, int num_sms);
cudaError_t launch_pack_f32(const Grid& g, const double* src, float2* dst, cudaStream_t s, int num_sms);
cudaError_t launch_unpack_f32(const Grid& g, const float2* src, double* dst, cudaStream_t s, int num_sms);
cudaError_t launch_unpack_elems(const Grid& g, const double* src, double* dst, cudaStream_t s,
                                int num_sms);
// Coarsest grid: z0 = K0^-1 b0 with the dense inverse (n x n, row-major).
template <typename T>
cudaError_t launch_coarsest_gemv(const Grid& g, int n, const int* free_idx, const double* Kinv,
                                 const typename V2<T>::t* b, typename V2<T>::t* z,
                                 DevScalars* sc, cudaStream_t s);
// Opt-in shared memory of the GEMV for n free coarsest DOFs (b is staged in
// shared memory: 8 n bytes), once per size, outside any stream capture.
cudaError_t prepare_coarsest_gemv(int n);
// Raises the opt-in dynamic shared memory limit of `func` on the current
// device to at least `bytes` (no call at 48 KiB or less).  The limit belongs
// to the kernel for the whole process, so it only ever grows: a context that
// needs less never lowers the limit another live context relies on.
// Thread-safe (one mutex for all kernels and devices).
cudaError_t raise_max_dynamic_smem(const void* func, size_t bytes);

// PCG scalars of a fresh solve; loop condition of the device-side solver loop;
// per-solve outcome record.
cudaError_t launch_init_scalars(DevScalars* sc, double tol2, int max_it, int flexible, int rr_every,
                                cudaStream_t s);
cudaError_t launch_set_continue(cudaGraphConditionalHandle h, const DevScalars* sc, cudaStream_t s);
cudaError_t launch_record_stats(const DevScalars* sc, RhsStats* dst, cudaStream_t s);

// ---- setup kernels (mto_setup.cu) ----
struct PhaseTable {
  double E[16];
};
// E_e = sum_i x_{e,i}^penal E_i (Eq. 5); ipenal >= 0 selects repeated products.
// Also writes E (kA, kB, kC, kG) per element (Ek4, 4 doubles) for the float64 sweeps.
// Element rows [j0, j1) (j1 < 0: to the last row).
cudaError_t launch_modulus(const Grid& g, int n_phase, const double* x, PhaseTable ph, double penal,
                           int ipenal, double* E64, __nv_bfloat16* Ebf, double* Ek4,
                           FineConst<double> kf, cudaStream_t s, int num_sms, int j0 = 0,
                           int j1 = -1);
// w / D on the float64 finest level (D = KE_00 * sum of the four moduli).
cudaError_t launch_fine_invd(const Grid& g, const double* E64, double w_over_kdiag, double* invd1,
                             cudaStream_t s, int num_sms);
// Moments of the first coarse level from the fine moduli (float64 or bf16).
cudaError_t launch_moments_from_fine(const Grid& gc, const Grid& gf, const double* E64,
                                     const __nv_bfloat16* Ebf, int rediscretize, double* mom,
                                     cudaStream_t s, int num_sms);
// Moments of level l-1 from those of level l.
cudaError_t launch_moments_from_coarse(const Grid& gc, const Grid& gf, const double* momf,
                                       int rediscretize, double* momc, cudaStream_t s, int num_sms);
template <typename T>
cudaError_t launch_coefs(const Grid& g, const double* mom, double nu, T* coef, cudaStream_t s,
                         int num_sms);
// w / D per DOF of a coarse level from its float64 element moments.
template <typename T>
cudaError_t launch_coarse_invd(const Grid& g, const double* mom, double nu, double omega,
                               typename V2<T>::t* invd2, cudaStream_t s, int num_sms);
// kappa-scaled float32 moments of a float32 coarse level (SRC_CMOM).
cudaError_t launch_kmom(const Grid& g, const double* mom, double nu, float* out, cudaStream_t s,
                        int num_sms);
// Coarsest matrix from float64 coefficients of level 0, lower band storage
// Kb[r * (bw + 1) + d] = K_0[r][r - d] (zeroed by the caller).
cudaError_t launch_band_assemble(const Grid& g, const double* coef64, const int* dof_index, int n,
                                 int bw, double* Kb, cudaStream_t s);
// Opt-in shared memory of the coarsest factorisation kernels (once per size,
// outside any stream capture).  Half-bandwidths up to MAX_COARSEST_BW keep
// the factorisation's index pairs (2 bw (bw + 1) bytes) and the inverse's
// ring (256 (bw + 1) bytes) within the opt-in shared memory of a block.
constexpr int MAX_COARSEST_BW = 320;
cudaError_t prepare_cholesky_inverse(int n, int bw);
// In-place band Cholesky of Kb (1 / L_ii to invL; the factor scaled by its
// columns' and rows' pivots to Lsc, 2 n (bw + 1) doubles), then the explicit
// inverse.
cudaError_t launch_cholesky_inverse(int n, int bw, double* Kb, double* invL, double* Lsc, double* Kinv,
                                    int* err_flag, cudaStream_t s, int num_sms);
// dcdx (+)= -penal x^(penal-1) E_i w_e, w_e = u_e^T KE u_e (dense user layouts),
// on element rows [j0, j1) (j1 < 0: to the last row).
cudaError_t launch_sensitivity(int nelx, int nely, int n_phase, const double* x, PhaseTable ph,
                               double penal, int ipenal, FineConst<double> kf, const double* u,
                               double* dcdx, int accumulate, cudaStream_t s, int num_sms, int j0 = 0,
                               int j1 = -1);

}  // namespace mto
