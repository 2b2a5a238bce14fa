// Shared device-side definitions of libmto: padded grid geometry, the Q4
// element operator in its strain basis, device scalars of the PCG recurrence
// and the deterministic block reduction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mto {

// Column index (inside a padded row) of node / element i = 0.  A multiple of
// 32 so that warps reading columns 0..31 start on a 256-byte boundary for
// float2 and a 512-byte boundary for double2.
constexpr int OFFX = 32;
// Entries of the symmetric 5x5 strain-basis element matrix that can be
// non-zero (see below).
constexpr int NCOEF = 13;
constexpr int NMOM = 6;

// Geometry of one grid level in the padded layout shared by its node and
// element arrays.  Node (i, j) and element (i, j) both live at
//   (j + 1) * pitch + OFFX + i,
// for i in [-OFFX, nx+65], j in [-1, ny+2]; everything outside the real mesh
// (ghost ring, right padding, extra rows) is zero and never written, so the
// stencil needs no bounds tests.
struct Grid {
  int nx, ny;      // elements in x and y
  int pitch;       // padded row length
  int rows;        // allocated rows (ny + 4)
  unsigned fixed;  // clamped-edge mask (MTO_EDGE_*)

  __host__ __device__ __forceinline__ long long at(int i, int j) const {
    return (long long)(j + 1) * pitch + OFFX + i;
  }
  __host__ __device__ __forceinline__ long long size() const { return (long long)rows * pitch; }
  __host__ __device__ __forceinline__ bool valid(int i, int j) const {
    return i >= 0 && i <= nx && j >= 0 && j <= ny;
  }
  __host__ __device__ __forceinline__ bool is_fixed(int i, int j) const {
    return ((fixed & 1u) && j == 0) || ((fixed & 2u) && i == 0) || ((fixed & 4u) && i == nx) ||
           ((fixed & 8u) && j == ny);
  }
  // A node whose DOFs the solver updates.
  __host__ __device__ __forceinline__ bool active(int i, int j) const {
    return valid(i, j) && !is_fixed(i, j);
  }
};

inline Grid make_grid(int nx, int ny, unsigned fixed) {
  Grid g;
  g.nx = nx;
  g.ny = ny;
  // Lanes of the marching sweeps read up to column nx + 62 (two columns per
  // lane) and down to column -2.
  g.pitch = ((OFFX + nx + 66) + 31) / 32 * 32;
  // Rows -1 .. ny + 3: the fused pre-smoothing and restriction marches two
  // rows past the last node row.
  g.rows = ny + 5;
  g.fixed = fixed;
  return g;
}

// Programmatic dependent launch.  The kernels of the PCG iteration are
// launched with launch_pdl (mto_launch.h): the next kernel on the stream may
// be scheduled while this one runs, and each of them calls pdl_wait() before
// its first global memory access, which returns once the previous grid has
// completed and its writes are visible.  The early trigger lets the next
// kernel's blocks take SM slots as this kernel's blocks retire, which hides
// the launch latency between the many short kernels of a V-cycle.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.launch_dependents;\n\tgriddepcontrol.wait;" ::: "memory");
}

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };

// Bit casts usable on the host (tests) and the device.
__host__ __device__ __forceinline__ unsigned long long bits_of(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &d, sizeof b);
  return b;
#endif
}
__host__ __device__ __forceinline__ double double_of(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, sizeof d);
  return d;
#endif
}
__host__ __device__ __forceinline__ unsigned bits_of(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned b;
  __builtin_memcpy(&b, &f, sizeof b);
  return b;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  __builtin_memcpy(&f, &b, sizeof f);
  return f;
#endif
}

// Conversions between float and double on the integer pipe.  On GB300 the
// FP64 pipe (two operations per clock per SM) also executes the hardware
// conversions, so kernels that are bound by that pipe, or that would become
// bound by it, convert here instead.
//
// f2d_exact: exact; normal numbers, zeros, infinities and NaNs keep their
// value; float subnormals (below 1.2e-38) become signed zero.
__host__ __device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = bits_of(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;  // rebias 127 -> 1023
  const unsigned hi = (b & 0x80000000u) | (e ? ((ed << 20) | ((b >> 3) & 0xfffffu)) : 0u);
  const unsigned lo = e ? (b << 29) : 0u;
  return double_of(((unsigned long long)hi << 32) | lo);
}
// d2f_rn: IEEE 754 round-to-nearest-even of the 52-bit significand to 23
// bits (ties to even).  Results below the float normal range (1.18e-38)
// become signed zero, overflow gives infinity, NaN stays NaN.
__host__ __device__ __forceinline__ float d2f_rn(double d) {
  const unsigned long long b = bits_of(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int fe = e - 896;                                  // rebias 1023 -> 127
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // leading 23 significand bits
  const unsigned half = (lo >> 28) & 1u;                   // first dropped bit
  const unsigned rest = lo & 0x0fffffffu;                  // the other dropped bits
  unsigned r = ((unsigned)fe << 23) + m;
  r += half & ((rest != 0u ? 1u : 0u) | (m & 1u));  // a carry moves into the exponent
  if (fe <= 0) r = 0u;
  if (fe >= 255) r = 0x7f800000u;
  if (e == 0x7ff) r = ((hi & 0xfffffu) | lo) != 0u ? 0x7fc00000u : 0x7f800000u;
  return float_of(sign | r);
}
__device__ __forceinline__ double to_f64(float f) { return f2d_exact(f); }
__device__ __forceinline__ double to_f64(double d) { return d; }

template <typename T> __device__ __forceinline__ typename V2<T>::t mk2(T x, T y) {
  typename V2<T>::t r;
  r.x = x;
  r.y = y;
  return r;
}

// ---------------------------------------------------------------------------
// Q4 element operator in the strain basis.
//
// On the reference square [-1,1]^2 a bilinear field is
//   u_x = c0 + c1 xi + c2 eta + c3 xi eta,  u_y = d0 + d1 xi + d2 eta + d3 xi eta,
// with (unscaled) c1 = -u0+u1+u2-u3, c2 = -u0-u1+u2+u3, c3 = u0-u1+u2-u3 for the
// nodes BL, BR, TR, TL (the same signs for d from u_y).  The strains are
//   eps_xx ~ c1 + c3 eta, eps_yy ~ d2 + d3 xi, gamma ~ (c2 + d1) + c3 xi + d3 eta,
// so the element energy u^T K_e u is a quadratic form in the five strain
// coordinates w = (c1, c3, d2, d3, s = c2 + d1) (the translations and the
// rotation c2 - d1 carry no energy).  Its symmetric 5x5 matrix A is linear in
// the moments M_ab = <E xi^a eta^b> of the modulus over the element:
//   A[c1,c1] = M00        A[c1,c3] = M01        A[c3,c3] = M02 + g M20
//   A[d2,d2] = M00        A[d2,d3] = M10        A[d3,d3] = M20 + g M02
//   A[c1,d2] = nu M00     A[c1,d3] = nu M10     A[c3,d2] = nu M01
//   A[c3,d3] = (nu+g) M11 A[s,s] = g M00        A[s,c3] = g M10   A[s,d3] = g M01
// all times kappa = 1 / (4 (1 - nu^2)) (plane stress, Eq. 8; g = (1-nu)/2).
// Then K_e v = J^T A J v, J the +-1 map above.  A unit-square fine element
// of modulus E has M = (E, 0, 0, E/3, E/3, 0); a Galerkin coarse element
// (P^T K P, nested bilinear spaces) has the moments of the fine moduli it
// covers, so every level uses the same operator.  The coefficient order in
// memory is the order of the table above read row by row:
//   0 c1c1, 1 c1c3, 2 c3c3, 3 d2d2, 4 d2d3, 5 d3d3, 6 c1d2, 7 c1d3, 8 c3d2,
//   9 c3d3, 10 ss, 11 c3s, 12 d3s.
// ---------------------------------------------------------------------------

template <typename T> struct Strain {
  T c1, c3, d2, d3, s;
};

// Strain coordinates of an element from its nodal values (BL, BR, TR, TL).
template <typename T, typename T2>
__device__ __forceinline__ Strain<T> strain_coords(const T2& bl, const T2& br, const T2& tr,
                                                   const T2& tl) {
  Strain<T> w;
  const T a = br.x - bl.x, b = tr.x - tl.x;    // bottom / top edge differences
  const T dl = tl.x - bl.x, dr = tr.x - br.x;  // left / right edge differences
  w.c1 = a + b;
  w.c3 = b - a;
  const T c2 = dl + dr;
  const T aw = br.y - bl.y, bw = tr.y - tl.y;
  const T dlw = tl.y - bl.y, drw = tr.y - br.y;
  const T d1 = aw + bw;
  w.d3 = bw - aw;
  w.d2 = dlw + drw;
  w.s = c2 + d1;
  return w;
}

// Nodal forces J^T t from the strain-space forces t (same basis as w).
template <typename T, typename T2>
__device__ __forceinline__ void strain_forces(const Strain<T>& t, T2& bl, T2& br, T2& tr, T2& tl) {
  const T ga = t.c1 - t.c3, gb = t.c1 + t.c3;
  bl.x = -ga - t.s;
  br.x = ga - t.s;
  tr.x = gb + t.s;
  tl.x = t.s - gb;
  const T gaw = t.s - t.d3, gbw = t.s + t.d3;
  bl.y = -gaw - t.d2;
  br.y = gaw - t.d2;
  tr.y = gbw + t.d2;
  tl.y = t.d2 - gbw;
}

// Fine element of modulus E: A = kappa E diag-structured.
template <typename T> struct FineConst {
  T kA, kB, kC, kG;  // kappa, kappa nu, kappa (1+g)/3, kappa g
};

template <typename T>
__device__ __forceinline__ Strain<T> fine_core(const Strain<T>& w, T E, const FineConst<T>& k) {
  const T eA = E * k.kA, eB = E * k.kB, eC = E * k.kC, eG = E * k.kG;
  Strain<T> t;
  t.c1 = eA * w.c1 + eB * w.d2;
  t.d2 = eA * w.d2 + eB * w.c1;
  t.c3 = eC * w.c3;
  t.d3 = eC * w.d3;
  t.s = eG * w.s;
  return t;
}

// The 13 coefficients of the table above from the six moments scaled by
// kappa, m = kappa (M00, M10, M01, M20, M02, M11), with nu and g = (1-nu)/2.
template <typename T>
__host__ __device__ __forceinline__ void coefs_from_kmom(const T m[NMOM], T nu, T g, T A[NCOEF]) {
  A[0] = m[0];
  A[1] = m[2];
  A[2] = m[4] + g * m[3];
  A[3] = m[0];
  A[4] = m[1];
  A[5] = m[3] + g * m[4];
  A[6] = nu * m[0];
  A[7] = nu * m[1];
  A[8] = nu * m[2];
  A[9] = (nu + g) * m[5];
  A[10] = g * m[0];
  A[11] = g * m[1];
  A[12] = g * m[2];
}

template <typename T>
__device__ __forceinline__ Strain<T> coarse_core(const Strain<T>& w, const T A[NCOEF]) {
  Strain<T> t;
  t.c1 = A[0] * w.c1 + A[1] * w.c3 + A[6] * w.d2 + A[7] * w.d3;
  t.c3 = A[1] * w.c1 + A[2] * w.c3 + A[8] * w.d2 + A[9] * w.d3 + A[11] * w.s;
  t.d2 = A[6] * w.c1 + A[8] * w.c3 + A[3] * w.d2 + A[4] * w.d3;
  t.d3 = A[7] * w.c1 + A[9] * w.c3 + A[4] * w.d2 + A[5] * w.d3 + A[12] * w.s;
  t.s = A[11] * w.c3 + A[12] * w.d3 + A[10] * w.s;
  return t;
}

// ---------------------------------------------------------------------------
// Device scalars of the PCG recurrence (Alg. 2).  Written only by the last
// block of a reduction kernel, read by the kernels that follow on the stream.
// ---------------------------------------------------------------------------
enum DoneCode { RUNNING = 0, CONVERGED = 1, MAXIT = 2, BREAKDOWN = 3 };

struct DevScalars {
  double rho;       // z_i . r_i
  double rho_prev;  // z_{i-1} . r_{i-1}
  double zq;        // z_i . q_{i-1} (flexible beta)
  double beta, alpha, pq;
  double rr;        // recursive ||r||^2
  double ff;        // ||f||^2 over free DOFs
  double tol2;      // tol^2
  double rr_true;   // ||f - K u||^2 (final check)
  double dot;       // scratch result of a plain dot kernel
  int iter, max_it, done, flexible, rr_every;
  int x_nonzero;    // set by the packing of the warm start when any entry is non-zero
  // The CG update applies r -= alpha q at once but x += alpha p one step
  // late, inside the next K p sweep (which loads p there anyway and is not
  // bound by memory): x_lag = 1 while x is one step behind, p_par says which
  // search-direction buffer holds that p.
  int x_lag, p_par;
  // Mixed precision: the update r -= alpha q of the last step is pending;
  // the next V-cycle's first smoothing sweep applies it (FIN_UPDATE_FUSED).
  int upd_pending;
};

// Outcome of one solve, copied from DevScalars at the end of each right-hand side.
struct RhsStats {
  int iter, done;
  double rr, rr_true, ff;
};

// Finishing actions of the last block of a reduction.
enum Finish {
  FIN_NONE = 0,
  FIN_DOT,        // sc->dot = s0
  FIN_FF,         // sc->ff = s0
  FIN_INIT_RR,    // sc->rr = s0; converged at start?
  FIN_RHO,        // sc->rho = s0 (, sc->zq = s1); beta
  FIN_PQ,         // sc->pq = s0; alpha
  FIN_UPDATE,     // sc->rr = s0; iter++; convergence
  FIN_REPLACE,    // sc->rr = s0 after residual replacement; convergence
  FIN_TRUE,       // sc->rr_true = s0
  FIN_PQ_FUSED,   // as FIN_PQ, and the step is complete but for r -= alpha q
  FIN_UPDATE_FUSED  // sc->rr = s0 after the fused r update, if one was pending
};

__device__ __forceinline__ bool finite_pos(double v) { return v > 0.0 && v < 1.0e300; }

__device__ __forceinline__ void finish_scalars(DevScalars* sc, int kind, double s0, double s1,
                                               int tag) {
  switch (kind) {
    case FIN_DOT: sc->dot = s0; break;
    case FIN_FF: sc->ff = s0; break;
    case FIN_INIT_RR:
      sc->rr = s0;
      if (!(s0 <= sc->tol2 * sc->ff)) {
        if (!(s0 < 1.0e300)) sc->done = BREAKDOWN;
      } else {
        sc->done = CONVERGED;
      }
      if (sc->done == RUNNING && sc->max_it <= 0) sc->done = MAXIT;
      break;
    case FIN_RHO: {
      sc->rho = s0;
      sc->zq = s1;
      if (!finite_pos(s0)) { sc->done = BREAKDOWN; break; }
      if (sc->iter == 0) sc->beta = 0.0;
      else if (sc->flexible) sc->beta = (-sc->alpha * s1) / sc->rho_prev;
      else sc->beta = s0 / sc->rho_prev;
      break;
    }
    case FIN_PQ:
      // The K p sweep has applied any pending x step; p[tag] is the new p.
      sc->x_lag = 0;
      sc->p_par = tag;
      sc->pq = s0;
      if (!finite_pos(s0)) { sc->done = BREAKDOWN; break; }
      sc->alpha = sc->rho / s0;
      break;
    case FIN_UPDATE: {
      sc->x_lag = 1;
      sc->rr = s0;
      sc->iter += 1;
      sc->rho_prev = sc->rho;
      const bool replace_now = sc->rr_every > 0 && (sc->iter % sc->rr_every) == 0;
      if (!(s0 < 1.0e300)) sc->done = BREAKDOWN;
      else if (!replace_now && s0 <= sc->tol2 * sc->ff) sc->done = CONVERGED;
      else if (!replace_now && sc->iter >= sc->max_it) sc->done = MAXIT;
      break;
    }
    case FIN_PQ_FUSED:
      // K p has applied any pending x step; with alpha known the new x step
      // and the r update are pending (applied by the next K p sweep and the
      // next V-cycle's first sweep), so the iteration is counted here.
      sc->x_lag = 0;
      sc->p_par = tag;
      sc->pq = s0;
      if (!finite_pos(s0)) { sc->done = BREAKDOWN; break; }
      sc->alpha = sc->rho / s0;
      sc->x_lag = 1;
      sc->upd_pending = 1;
      sc->rho_prev = sc->rho;
      sc->iter += 1;
      break;
    case FIN_UPDATE_FUSED:
      if (!sc->upd_pending) break;  // the residual was replaced instead
      sc->upd_pending = 0;
      sc->rr = s0;
      if (!(s0 < 1.0e300)) sc->done = BREAKDOWN;
      else if (s0 <= sc->tol2 * sc->ff) sc->done = CONVERGED;
      else if (sc->iter >= sc->max_it) sc->done = MAXIT;
      break;
    case FIN_REPLACE:
      sc->upd_pending = 0;
      sc->rr = s0;
      if (!(s0 < 1.0e300)) sc->done = BREAKDOWN;
      else if (s0 <= sc->tol2 * sc->ff) sc->done = CONVERGED;
      else if (sc->iter >= sc->max_it) sc->done = MAXIT;
      break;
    case FIN_TRUE: sc->rr_true = s0; break;
    default: break;
  }
}

// Deterministic two-stage sum of up to two values per thread.  Every thread
// of the block must call it.  Block partials go to partials[2*blockIdx.x + k];
// the last block to arrive (ticket) adds them in block order, runs the
// finishing action and re-arms the ticket.  No floating-point atomics.
template <int NT>
__device__ __forceinline__ void block_reduce_finish(double v0, double v1, double* partials,
                                                    unsigned* ticket, DevScalars* sc, int kind,
                                                    double* out_value, int tag = 0) {
  __shared__ double red[2][NT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  if (lane == 0) {
    red[0][wid] = v0;
    red[1][wid] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // Last block: sum the partials in block order (fixed for a fixed grid).
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += NT) {
    a += ((volatile double*)partials)[2 * k];
    b += ((volatile double*)partials)[2 * k + 1];
  }
  // Fixed-order tree over the block's threads.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    if (sc) finish_scalars(sc, kind, s0, s1, tag);
    if (out_value) out_value[0] = s0;
    *ticket = 0u;
    __threadfence();
  }
}

}  // namespace mto
