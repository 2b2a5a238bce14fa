// Pointwise kernels of the PCG recurrence (Alg. 2), the first smoothing sweep
// from a zero iterate (Sec. 2.3 with x_0 = 0), layout conversions and the
// coarsest-grid solve of Alg. 1 (l = 0) as a dense product with K_0^-1.
#include <map>
#include <mutex>
#include <utility>

#include "mto_gemv.cuh"
#include "mto_launch.h"

namespace mto {

thread_local bool g_pdl = true;

int vec_blocks(long long n, int num_sms) {
  long long b = (n + VEC_NT - 1) / VEC_NT;
  const long long cap = (long long)num_sms * 8;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

__device__ __forceinline__ void node_of(const Grid& g, long long k, int& i, int& j) {
  j = (int)(k / g.pitch) - 1;
  i = (int)(k - (long long)(j + 1) * g.pitch) - OFFX;
}

__device__ __forceinline__ bool stop_now(const DevScalars* sc) {
  return sc != nullptr && sc->done != RUNNING;
}

__global__ void jacobi0_fine64_kernel(Grid g, const double* __restrict__ invd1,
                                      const double2* __restrict__ r, double2* __restrict__ z,
                                      const DevScalars* sc) {
  pdl_wait();
  if (stop_now(sc)) return;
  const long long n = g.size();
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    int i, j;
    node_of(g, k, i, j);
    double2 out = make_double2(0.0, 0.0);
    if (g.active(i, j)) {
      const double d = invd1[k];
      const double2 rr = r[k];
      out = make_double2(d * rr.x, d * rr.y);
    }
    z[k] = out;
  }
}

__global__ void jacobi0_finebf_kernel(Grid g, const __nv_bfloat16* __restrict__ E, float wdiag,
                                      const float2* __restrict__ r32, float2* __restrict__ z,
                                      const DevScalars* sc) {
  pdl_wait();
  if (stop_now(sc)) return;
  const long long n = g.size();
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    int i, j;
    node_of(g, k, i, j);
    float2 out = make_float2(0.f, 0.f);
    if (g.active(i, j)) {
      const float2 rf = r32[k];
      const float se = __bfloat162float(E[k]) + __bfloat162float(E[k - 1]) +
                       __bfloat162float(E[k - g.pitch]) + __bfloat162float(E[k - g.pitch - 1]);
      const float d = __fdividef(wdiag, se);
      out = make_float2(d * rf.x, d * rf.y);
    }
    z[k] = out;
  }
}

template <typename T>
__global__ void jacobi0_coarse_kernel(Grid g, const typename V2<T>::t* __restrict__ invd2,
                                      const typename V2<T>::t* __restrict__ b,
                                      typename V2<T>::t* __restrict__ z, const DevScalars* sc) {
  pdl_wait();
  if (stop_now(sc)) return;
  const long long n = g.size();
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    int i, j;
    node_of(g, k, i, j);
    typename V2<T>::t out = mk2<T>(T(0), T(0));
    if (g.active(i, j)) {
      const typename V2<T>::t d = invd2[k], bb = b[k];
      out = mk2<T>(d.x * bb.x, d.y * bb.y);
    }
    z[k] = out;
  }
}

// r -= alpha q, |r|^2 (FIN_UPDATE, which marks the x step as pending), and
// the float32 copy of r.  x += alpha p happens in the next K p sweep or in
// x_step_kernel after the loop.
__global__ void __launch_bounds__(VEC_NT)
    update_kernel(long long n, double2* __restrict__ r, float2* __restrict__ r32,
                  const double2* __restrict__ q, double* partials, unsigned* ticket,
                  DevScalars* sc) {
  pdl_wait();
  if (sc->done != RUNNING) return;
  const double alpha = sc->alpha;
  double acc = 0.0;
  auto one = [&](long long k, const double2 qq, double2 rr) {
    rr.x -= alpha * qq.x;
    rr.y -= alpha * qq.y;
    r[k] = rr;
    if (r32 != nullptr) r32[k] = make_float2(d2f_rn(rr.x), d2f_rn(rr.y));
    acc = fma(rr.x, rr.x, fma(rr.y, rr.y, acc));
  };
  // Two nodes per pass with the loads issued first (more bytes in flight).
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + stride < n; k += 2 * stride) {
    const double2 q0 = q[k], r0 = r[k], q1 = q[k + stride], r1 = r[k + stride];
    one(k, q0, r0);
    one(k + stride, q1, r1);
  }
  if (k < n) one(k, q[k], r[k]);
  block_reduce_finish<VEC_NT>(acc, 0.0, partials, ticket, sc, FIN_UPDATE, nullptr);
}

// The pending x step after the loop: x += alpha p[p_par] when x_lag.
__global__ void __launch_bounds__(VEC_NT)
    x_step_kernel(long long n, double2* __restrict__ x, const double2* __restrict__ p0,
                  const double2* __restrict__ p1, const DevScalars* sc) {
  pdl_wait();
  if (sc->x_lag == 0) return;
  const double alpha = sc->alpha;
  const double2* __restrict__ p = sc->p_par ? p1 : p0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const double2 pp = p[k];
    double2 xx = x[k];
    xx.x = fma(alpha, pp.x, xx.x);
    xx.y = fma(alpha, pp.y, xx.y);
    x[k] = xx;
  }
}

__global__ void __launch_bounds__(VEC_NT)
    dot_kernel(long long n, const double2* __restrict__ a, const double2* __restrict__ b,
               double* partials, unsigned* ticket, DevScalars* sc, int finish, double* out_value) {
  pdl_wait();
  // Two nodes per pass into two FMA chains, the loads issued first.
  double acc0 = 0.0, acc1 = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + stride < n; k += 2 * stride) {
    const double2 x0 = a[k], y0 = b[k], x1 = a[k + stride], y1 = b[k + stride];
    acc0 = fma(x0.x, y0.x, fma(x0.y, y0.y, acc0));
    acc1 = fma(x1.x, y1.x, fma(x1.y, y1.y, acc1));
  }
  if (k < n) {
    const double2 x = a[k], y = b[k];
    acc0 = fma(x.x, y.x, fma(x.y, y.y, acc0));
  }
  block_reduce_finish<VEC_NT>(acc0 + acc1, 0.0, partials, ticket, sc, finish, out_value);
}

__global__ void pack_kernel(Grid g, const double* __restrict__ src, double2* __restrict__ dst,
                            int* nonzero) {
  const long long n = g.size();
  bool nz = false;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    int i, j;
    node_of(g, k, i, j);
    double2 v = make_double2(0.0, 0.0);
    if (g.active(i, j)) {
      const long long s = 2 * ((long long)j * (g.nx + 1) + i);
      v = make_double2(src[s], src[s + 1]);
      nz = nz || v.x != 0.0 || v.y != 0.0;
    }
    dst[k] = v;
  }
  if (nonzero != nullptr && __any_sync(0xffffffffu, nz) && (threadIdx.x & 31) == 0) atomicOr(nonzero, 1);
}

__global__ void unpack_kernel(Grid g, const double2* __restrict__ src, double* __restrict__ dst) {
  const long long n = (long long)(g.nx + 1) * (g.ny + 1);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k % (g.nx + 1)), j = (int)(k / (g.nx + 1));
    const double2 v = src[g.at(i, j)];
    dst[2 * k] = v.x;
    dst[2 * k + 1] = v.y;
  }
}

__global__ void pack_f32_kernel(Grid g, const double* __restrict__ src, float2* __restrict__ dst) {
  const long long n = g.size();
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    int i, j;
    node_of(g, k, i, j);
    float2 v = make_float2(0.f, 0.f);
    if (g.active(i, j)) {
      const long long s = 2 * ((long long)j * (g.nx + 1) + i);
      v = make_float2((float)src[s], (float)src[s + 1]);
    }
    dst[k] = v;
  }
}

__global__ void unpack_f32_kernel(Grid g, const float2* __restrict__ src, double* __restrict__ dst) {
  const long long n = (long long)(g.nx + 1) * (g.ny + 1);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k % (g.nx + 1)), j = (int)(k / (g.nx + 1));
    const float2 v = src[g.at(i, j)];
    dst[2 * k] = v.x;
    dst[2 * k + 1] = v.y;
  }
}

__global__ void unpack_elems_kernel(Grid g, const double* __restrict__ src, double* __restrict__ dst) {
  const long long n = (long long)g.nx * g.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    dst[k] = src[g.at((int)(k % g.nx), (int)(k / g.nx))];
  }
}

// One warp per row of K_0^-1; every block stages the free coarse right-hand
// side in shared memory first (mto_gemv.cuh).
constexpr int GEMV_NT = 256;

template <typename T>
__global__ void __launch_bounds__(GEMV_NT)
    coarsest_gemv_kernel(int n, const int* __restrict__ free_idx, const double* __restrict__ Kinv,
                         const T* __restrict__ b, T* __restrict__ z, const DevScalars* sc) {
  // K_0^-1 and the DOF map are set up once per design: load this warp's row
  // before waiting for the previous kernel (programmatic dependent launch).
  const int row = blockIdx.x * (GEMV_NT / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  double kreg[GEMV_REG_COLS];
  int zidx = 0;
  if (row < n) gemv_prefetch(n, row, lane, free_idx, Kinv, kreg, zidx);
  pdl_wait();
  if (stop_now(sc)) return;
  extern __shared__ double bs[];
  gemv_stage<T>(n, free_idx, b, bs);
  if (row < n) gemv_row<T>(n, row, lane, free_idx, Kinv, bs, z, kreg, zidx);
}

// PCG scalars of a fresh solve (kernel parameters, so the launch can live in a
// CUDA graph).
__global__ void init_scalars_kernel(DevScalars* sc, double tol2, int max_it, int flexible,
                                    int rr_every) {
  DevScalars s;
  memset(&s, 0, sizeof(s));
  s.tol2 = tol2;
  s.max_it = max_it;
  s.flexible = flexible;
  s.rr_every = rr_every;
  *sc = s;
}

// Body condition of the solver's device-side loop: run again while the PCG
// has not stopped.
__global__ void set_continue_kernel(cudaGraphConditionalHandle h, const DevScalars* sc) {
  pdl_wait();
  cudaGraphSetConditional(h, sc->done == RUNNING ? 1u : 0u);
}

__global__ void record_stats_kernel(const DevScalars* sc, RhsStats* dst) {
  RhsStats r;
  r.iter = sc->iter;
  r.done = sc->done;
  r.rr = sc->rr;
  r.rr_true = sc->rr_true;
  r.ff = sc->ff;
  *dst = r;
}

// ---------------------------------------------------------------------------

cudaError_t launch_init_scalars(DevScalars* sc, double tol2, int max_it, int flexible, int rr_every,
                                cudaStream_t s) {
  init_scalars_kernel<<<1, 1, 0, s>>>(sc, tol2, max_it, flexible, rr_every);
  return cudaGetLastError();
}

cudaError_t launch_set_continue(cudaGraphConditionalHandle h, const DevScalars* sc, cudaStream_t s) {
  return launch_pdl(set_continue_kernel, 1, 1, 0, s, h, sc);
}

cudaError_t launch_record_stats(const DevScalars* sc, RhsStats* dst, cudaStream_t s) {
  record_stats_kernel<<<1, 1, 0, s>>>(sc, dst);
  return cudaGetLastError();
}

cudaError_t launch_jacobi0_fine64(const Grid& g, const double* invd1, const double2* r, double2* z,
                                  DevScalars* sc, int nblocks, cudaStream_t s) {
  return launch_pdl(jacobi0_fine64_kernel, nblocks, VEC_NT, 0, s, g, invd1, r, z, sc);
}

cudaError_t launch_jacobi0_finebf(const Grid& g, const __nv_bfloat16* E, float wdiag,
                                  const float2* r32, float2* z, DevScalars* sc, int nblocks,
                                  cudaStream_t s) {
  return launch_pdl(jacobi0_finebf_kernel, nblocks, VEC_NT, 0, s, g, E, wdiag, r32, z, sc);
}

template <typename T>
cudaError_t launch_jacobi0_coarse(const Grid& g, const typename V2<T>::t* invd2,
                                  const typename V2<T>::t* b, typename V2<T>::t* z,
                                  DevScalars* sc, int nblocks, cudaStream_t s) {
  return launch_pdl(jacobi0_coarse_kernel<T>, nblocks, VEC_NT, 0, s, g, invd2, b, z, sc);
}
template cudaError_t launch_jacobi0_coarse<double>(const Grid&, const double2*, const double2*,
                                                   double2*, DevScalars*, int, cudaStream_t);
template cudaError_t launch_jacobi0_coarse<float>(const Grid&, const float2*, const float2*,
                                                  float2*, DevScalars*, int, cudaStream_t);

cudaError_t launch_update(const Grid& g, double2* r, float2* r32, const double2* q,
                          double* partials, unsigned* ticket, DevScalars* sc, int nblocks,
                          cudaStream_t s) {
  return launch_pdl(update_kernel, nblocks, VEC_NT, 0, s, g.size(), r, r32, q, partials, ticket, sc);
}

cudaError_t launch_x_step(const Grid& g, double2* x, const double2* p0, const double2* p1,
                          const DevScalars* sc, int nblocks, cudaStream_t s) {
  return launch_pdl(x_step_kernel, nblocks, VEC_NT, 0, s, g.size(), x, p0, p1, sc);
}

cudaError_t launch_dot(long long n, const double2* a, const double2* b, double* partials,
                       unsigned* ticket, DevScalars* sc, int finish, double* out_value,
                       int nblocks, cudaStream_t s) {
  return launch_pdl(dot_kernel, nblocks, VEC_NT, 0, s, n, a, b, partials, ticket, sc, finish, out_value);
}

cudaError_t launch_pack(const Grid& g, const double* src, double2* dst, cudaStream_t s, int num_sms,
                        int* nonzero) {
  pack_kernel<<<vec_blocks(g.size(), num_sms), VEC_NT, 0, s>>>(g, src, dst, nonzero);
  return cudaGetLastError();
}
cudaError_t launch_unpack(const Grid& g, const double2* src, double* dst, cudaStream_t s, int num_sms) {
  unpack_kernel<<<vec_blocks((long long)(g.nx + 1) * (g.ny + 1), num_sms), VEC_NT, 0, s>>>(g, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_pack_f32(const Grid& g, const double* src, float2* dst, cudaStream_t s, int num_sms) {
  pack_f32_kernel<<<vec_blocks(g.size(), num_sms), VEC_NT, 0, s>>>(g, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_unpack_f32(const Grid& g, const float2* src, double* dst, cudaStream_t s, int num_sms) {
  unpack_f32_kernel<<<vec_blocks((long long)(g.nx + 1) * (g.ny + 1), num_sms), VEC_NT, 0, s>>>(g, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_unpack_elems(const Grid& g, const double* src, double* dst, cudaStream_t s,
                                int num_sms) {
  unpack_elems_kernel<<<vec_blocks((long long)g.nx * g.ny, num_sms), VEC_NT, 0, s>>>(g, src, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsest_gemv(const Grid& g, int n, const int* free_idx, const double* Kinv,
                                 const typename V2<T>::t* b, typename V2<T>::t* z,
                                 DevScalars* sc, cudaStream_t s) {
  (void)g;
  if (n > GEMV_MAXN) return cudaErrorInvalidValue;
  const int blocks = (n + GEMV_NT / 32 - 1) / (GEMV_NT / 32);
  return launch_pdl(coarsest_gemv_kernel<T>, blocks, GEMV_NT, n * sizeof(double), s, n, free_idx, Kinv,
                    reinterpret_cast<const T*>(b), reinterpret_cast<T*>(z),
                    static_cast<const DevScalars*>(sc));
}
cudaError_t raise_max_dynamic_smem(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> current;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = current[{dev, func}];
  if (bytes <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

cudaError_t prepare_coarsest_gemv(int n) {
  if (n > GEMV_MAXN) return cudaErrorInvalidValue;
  const size_t bytes = (size_t)n * sizeof(double);
  cudaError_t e = raise_max_dynamic_smem((const void*)coarsest_gemv_kernel<double>, bytes);
  if (e != cudaSuccess) return e;
  return raise_max_dynamic_smem((const void*)coarsest_gemv_kernel<float>, bytes);
}

template cudaError_t launch_coarsest_gemv<double>(const Grid&, int, const int*, const double*,
                                                  const double2*, double2*, DevScalars*, cudaStream_t);
template cudaError_t launch_coarsest_gemv<float>(const Grid&, int, const int*, const double*,
                                                 const float2*, float2*, DevScalars*, cudaStream_t);

}  // namespace mto
