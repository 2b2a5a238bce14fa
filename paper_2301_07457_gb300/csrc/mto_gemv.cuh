// Coarsest-level solve z = K_0^-1 b as a dense float64 GEMV (Alg. 1 on the
// coarsest grid, Alg. 3 factor turned into an explicit inverse at setup).
// Device functions of the coarsest GEMV kernel (mto_vec.cu).
#pragma once

#include "mto_common.cuh"

namespace mto {

// Largest coarsest system: b is staged in shared memory (132 KiB at the
// limit; the kernel opts in above 48 KiB), and K_0^-1 takes 8 n^2 bytes
// (2.3 GB at the limit).
constexpr int GEMV_MAXN = 16896;

// Every thread of the block: stage b at the free DOFs in shared memory
// (free_idx[k] = scalar index 2 * node offset + component of free DOF k).
template <typename T>
__device__ __forceinline__ void gemv_stage(int n, const int* __restrict__ free_idx,
                                           const T* __restrict__ b, double* bs) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) bs[k] = (double)b[free_idx[k]];
  __syncthreads();
}

// Entries of a K_0^-1 row one lane holds in registers (lane, lane + 32, ...):
// n <= GEMV_REG_COLS * 32 rows use the register path, larger ones read the
// row from memory after the wait.
constexpr int GEMV_REG_COLS = 24;

// One warp: row `row` of K_0^-1 times the staged b, written to z at the free
// DOF (fixed DOFs of z stay zero).  kreg holds the lane's entries of the row
// when n <= 32 GEMV_REG_COLS (loaded before the wait for the previous kernel,
// since K_0^-1 and the DOF map do not depend on it).
template <typename T>
__device__ __forceinline__ void gemv_row(int n, int row, int lane, const int* __restrict__ free_idx,
                                         const double* __restrict__ Kinv, const double* bs,
                                         T* __restrict__ z, const double* kreg, int zidx) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;  // independent chains
  if (n <= GEMV_REG_COLS * 32) {
#pragma unroll
    for (int c = 0; c < GEMV_REG_COLS; c += 4) {
      const int k = lane + 32 * c;
      if (k < n) a0 = fma(kreg[c], bs[k], a0);
      if (k + 32 < n) a1 = fma(kreg[c + 1], bs[k + 32], a1);
      if (k + 64 < n) a2 = fma(kreg[c + 2], bs[k + 64], a2);
      if (k + 96 < n) a3 = fma(kreg[c + 3], bs[k + 96], a3);
    }
  } else {
    const double* kr = Kinv + (long long)row * n;
    int k = lane;
    for (; k + 96 < n; k += 128) {
      a0 = fma(kr[k], bs[k], a0);
      a1 = fma(kr[k + 32], bs[k + 32], a1);
      a2 = fma(kr[k + 64], bs[k + 64], a2);
      a3 = fma(kr[k + 96], bs[k + 96], a3);
    }
    for (; k < n; k += 32) a0 = fma(kr[k], bs[k], a0);
  }
  double acc = (a0 + a1) + (a2 + a3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) z[zidx] = (T)acc;
  (void)free_idx;
}

// The lane's entries of row `row` (register path) and the row's DOF index.
__device__ __forceinline__ void gemv_prefetch(int n, int row, int lane, const int* __restrict__ free_idx,
                                              const double* __restrict__ Kinv, double* kreg,
                                              int& zidx) {
  zidx = free_idx[row];
  if (n <= GEMV_REG_COLS * 32) {
    const double* kr = Kinv + (long long)row * n;
#pragma unroll
    for (int c = 0; c < GEMV_REG_COLS; ++c) {
      const int k = lane + 32 * c;
      kreg[c] = k < n ? kr[k] : 0.0;
    }
  }
}

}  // namespace mto
