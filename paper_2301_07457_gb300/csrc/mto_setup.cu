// Per-design setup of the level hierarchy and the compliance sensitivities:
//   * element moduli E_e = sum_i x_{e,i}^p E_i (Eq. 5), float64 and bfloat16;
//   * the Jacobi diagonal D of the finest level (Sec. 2.3);
//   * coarse operators: Galerkin moments of the fine moduli per coarse
//     element (exact P^T K P for nested bilinear spaces) or the rediscretised
//     mean modulus (Sec. 2.1), their 13 strain-basis coefficients and the
//     Jacobi diagonals of every coarse level;
//   * the coarsest grid (Alg. 1, l = 0): K_0 on the free DOFs in band
//     storage, its Cholesky factor (Alg. 3), and the explicit K_0^-1;
//   * sensitivities dC/dx_{e,i} = -p x^{p-1} E_i u_e^T KE u_e (Eq. 6, Sec. 4).
#include "mto_launch.h"

namespace mto {

__device__ __forceinline__ double xpow(double x, double p, int ip) {
  if (ip >= 0) {
    double r = 1.0;
    for (int k = 0; k < ip; ++k) r *= x;
    return r;
  }
  return pow(x, p);
}

// Element rows [j0, j1).
__global__ void modulus_kernel(Grid g, int j0, int j1, int n_phase, const double* __restrict__ x,
                               PhaseTable ph, double penal, int ipenal, double* __restrict__ E64,
                               __nv_bfloat16* __restrict__ Ebf, double* __restrict__ Ek4,
                               FineConst<double> kf) {
  const long long n = (long long)g.nx * g.ny;
  const long long e1 = (long long)j1 * g.nx;
  for (long long e = (long long)j0 * g.nx + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < e1;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.nx), j = (int)(e / g.nx);
    double E = 0.0;
    for (int p = 0; p < n_phase; ++p) E += ph.E[p] * xpow(x[(long long)p * n + e], penal, ipenal);
    const long long k = g.at(i, j);
    E64[k] = E;
    if (Ebf) Ebf[k] = __double2bfloat16(E);
    // The fine element core's four scale factors, stored so that the float64
    // sweeps spend no FP64 multiplies on them.
    double2* q = reinterpret_cast<double2*>(Ek4) + 2 * k;
    q[0] = make_double2(E * kf.kA, E * kf.kB);
    q[1] = make_double2(E * kf.kC, E * kf.kG);
  }
}

__global__ void fine_invd_kernel(Grid g, const double* __restrict__ E, double w_over_kdiag,
                                 double* __restrict__ invd1) {
  const long long n = (long long)(g.nx + 1) * (g.ny + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % (g.nx + 1)), j = (int)(t / (g.nx + 1));
    const long long k = g.at(i, j);
    double d = 0.0;
    if (!g.is_fixed(i, j)) {
      const double se = ((E[k - g.pitch - 1] + E[k - g.pitch]) + E[k - 1]) + E[k];
      d = w_over_kdiag / se;
    }
    invd1[k] = d;
  }
}

// Moments M_ab = <E xi^a eta^b> (a + b <= 2) of a parent element from its four
// children, each child mapped by xi = (xi' + sx) / 2, eta = (eta' + sy) / 2.
struct Mom {
  double m00, m10, m01, m20, m02, m11;
};

__device__ __forceinline__ void accum_child(Mom& P, const Mom& c, double sx, double sy) {
  P.m00 += 0.25 * c.m00;
  P.m10 += 0.125 * (c.m10 + sx * c.m00);
  P.m01 += 0.125 * (c.m01 + sy * c.m00);
  P.m20 += 0.0625 * (c.m20 + 2.0 * sx * c.m10 + c.m00);
  P.m02 += 0.0625 * (c.m02 + 2.0 * sy * c.m01 + c.m00);
  P.m11 += 0.0625 * (c.m11 + sy * c.m10 + sx * c.m01 + sx * sy * c.m00);
}

__device__ __forceinline__ void store_mom(double* mom, long long stride, long long k, const Mom& M) {
  mom[0 * stride + k] = M.m00;
  mom[1 * stride + k] = M.m10;
  mom[2 * stride + k] = M.m01;
  mom[3 * stride + k] = M.m20;
  mom[4 * stride + k] = M.m02;
  mom[5 * stride + k] = M.m11;
}

__global__ void moments_from_fine_kernel(Grid gc, Grid gf, const double* __restrict__ E64,
                                         const __nv_bfloat16* __restrict__ Ebf, int redisc,
                                         double* __restrict__ mom) {
  const long long n = (long long)gc.nx * gc.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % gc.nx), J = (int)(t / gc.nx);
    // Children of constant modulus at xi, eta = +-1/2: the shift-and-scale
    // rule of accum_child in closed form, M00 = S/4, M10 = X/8, M01 = Y/8,
    // M20 = M02 = M00/3, M11 = Z/16 (S, X, Y, Z: sums of the child moduli
    // with signs 1, s_x, s_y, s_x s_y).
    const long long kf = gf.at(2 * I, 2 * J);
    double e[2][2];
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const long long k = kf + (long long)cy * gf.pitch + cx;
        e[cy][cx] = Ebf ? (double)__bfloat162float(Ebf[k]) : E64[k];
      }
    const double S = (e[0][0] + e[0][1]) + (e[1][0] + e[1][1]);
    const double M00 = 0.25 * S;
    Mom P = {M00, 0.0, 0.0, M00 / 3.0, M00 / 3.0, 0.0};
    if (!redisc) {
      P.m10 = 0.125 * ((e[0][1] + e[1][1]) - (e[0][0] + e[1][0]));
      P.m01 = 0.125 * ((e[1][0] + e[1][1]) - (e[0][0] + e[0][1]));
      P.m11 = 0.0625 * ((e[0][0] + e[1][1]) - (e[0][1] + e[1][0]));
    }
    store_mom(mom, gc.size(), gc.at(I, J), P);
  }
}

__global__ void moments_from_coarse_kernel(Grid gc, Grid gf, const double* __restrict__ momf,
                                           int redisc, double* __restrict__ momc) {
  const long long n = (long long)gc.nx * gc.ny;
  const long long sf = gf.size();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % gc.nx), J = (int)(t / gc.nx);
    Mom P = {0, 0, 0, 0, 0, 0};
    double Emean = 0.0;
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const long long kf = gf.at(2 * I + cx, 2 * J + cy);
        const Mom c = {momf[kf], momf[sf + kf], momf[2 * sf + kf],
                       momf[3 * sf + kf], momf[4 * sf + kf], momf[5 * sf + kf]};
        accum_child(P, c, 2.0 * cx - 1.0, 2.0 * cy - 1.0);
        Emean += 0.25 * c.m00;
      }
    if (redisc) P = {Emean, 0.0, 0.0, Emean / 3.0, Emean / 3.0, 0.0};
    store_mom(momc, gc.size(), gc.at(I, J), P);
  }
}

template <typename T>
__global__ void coefs_kernel(Grid g, const double* __restrict__ mom, double nu, T* __restrict__ coef) {
  const long long n = (long long)g.nx * g.ny;
  const long long s = g.size();
  const double kap = 1.0 / (4.0 * (1.0 - nu * nu)), gs = 0.5 * (1.0 - nu);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % g.nx), J = (int)(t / g.nx);
    const long long k = g.at(I, J);
    const double M00 = mom[k], M10 = mom[s + k], M01 = mom[2 * s + k];
    const double M20 = mom[3 * s + k], M02 = mom[4 * s + k], M11 = mom[5 * s + k];
    const double A[NCOEF] = {kap * M00,           kap * M01,       kap * (M02 + gs * M20),
                             kap * M00,           kap * M10,       kap * (M20 + gs * M02),
                             kap * nu * M00,      kap * nu * M10,  kap * nu * M01,
                             kap * (nu + gs) * M11, kap * gs * M00, kap * gs * M10,
                             kap * gs * M01};
#pragma unroll
    for (int c = 0; c < NCOEF; ++c) coef[c * s + k] = (T)A[c];
  }
}

// Diagonal of an element matrix J^T A J at local node q (0 BL, 1 BR, 2 TR, 3 TL):
// J column of u_x at q is (s1, s3, 0, 0, s2), of u_y is (0, 0, s2, s3, s1), with
// s1 = (-1, 1, 1, -1), s2 = (-1, -1, 1, 1), s3 = (1, -1, 1, -1); s1 s3 = s2, s2 s3 = s1.
template <typename C>
__device__ __forceinline__ void elem_diag(const C A[NCOEF], int q, C& dx, C& dy) {
  const C s1 = (q == 1 || q == 2) ? C(1) : C(-1);
  const C s2 = (q >= 2) ? C(1) : C(-1);
  dx += A[0] + A[2] + A[10] + C(2) * s2 * A[1] + C(2) * s1 * A[11];
  dy += A[3] + A[5] + A[10] + C(2) * s1 * A[4] + C(2) * s2 * A[12];
}

// Coefficients of element k from the float64 moments (zero for ghost
// elements), in the precision C of the level (float32 levels convert the
// moments on the integer pipe and stay off the FP64 pipe).
template <typename C>
__device__ __forceinline__ void coefs_at(const double* __restrict__ mom, long long s, long long k,
                                         C kap, C nu, C gs, C A[NCOEF]) {
  C m[NMOM];
#pragma unroll
  for (int c = 0; c < NMOM; ++c) {
    if constexpr (sizeof(C) == 4) m[c] = kap * d2f_rn(mom[c * s + k]);
    else m[c] = kap * mom[c * s + k];
  }
  coefs_from_kmom<C>(m, nu, gs, A);
}

// w / D per DOF of a coarse level, from the moments of its elements.
template <typename T>
__global__ void coarse_invd_kernel(Grid g, const double* __restrict__ mom, double nu, double omega,
                                   typename V2<T>::t* __restrict__ invd2) {
  const long long n = (long long)(g.nx + 1) * (g.ny + 1);
  const long long s = g.size();
  const T kap = T(1.0 / (4.0 * (1.0 - nu * nu))), gs = T(0.5 * (1.0 - nu)), nut = T(nu);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % (g.nx + 1)), j = (int)(t / (g.nx + 1));
    const long long k = g.at(i, j);
    typename V2<T>::t out = mk2<T>(T(0), T(0));
    if (!g.is_fixed(i, j)) {
      T dx = T(0), dy = T(0), A[NCOEF];
      // Ghost elements have zero moments, so all four may be visited.
      coefs_at<T>(mom, s, k - g.pitch - 1, kap, nut, gs, A);
      elem_diag<T>(A, 2, dx, dy);  // element (i-1, j-1): node is TR
      coefs_at<T>(mom, s, k - g.pitch, kap, nut, gs, A);
      elem_diag<T>(A, 3, dx, dy);  // element (i, j-1): TL
      coefs_at<T>(mom, s, k - 1, kap, nut, gs, A);
      elem_diag<T>(A, 1, dx, dy);  // element (i-1, j): BR
      coefs_at<T>(mom, s, k, kap, nut, gs, A);
      elem_diag<T>(A, 0, dx, dy);  // element (i, j): BL
      out = mk2<T>(T(omega) / dx, T(omega) / dy);
    }
    invd2[k] = out;
  }
}

// Six kappa-scaled float32 moments per element of a float32 coarse level
// (SRC_CMOM sweeps).
__global__ void kmom_kernel(Grid g, const double* __restrict__ mom, double nu, float* __restrict__ out) {
  const long long n = (long long)g.nx * g.ny;
  const long long s = g.size();
  const double kap = 1.0 / (4.0 * (1.0 - nu * nu));
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % g.nx), J = (int)(t / g.nx);
    const long long k = g.at(I, J);
#pragma unroll
    for (int c = 0; c < NMOM; ++c) out[c * s + k] = (float)(kap * mom[c * s + k]);
  }
}

// Row r of the coarsest matrix K_0 (free DOF (node (i, j), component c)) in
// lower band storage: Kb[r * (bw + 1) + d] = K_0[r][r - d], d = 0..bw.
__global__ void band_assemble_kernel(Grid g, const double* __restrict__ coef,
                                     const int* __restrict__ dof_index, int n, int bw,
                                     double* __restrict__ Kb) {
  const long long s = g.size();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    // Find the node of row r: scan is avoided by storing the inverse map in
    // dof_index's second half (2 * g.size() .. + n).
    const int sidx = dof_index[2 * s + r];
    const long long k = sidx >> 1;
    const int c = sidx & 1;
    const int j = (int)(k / g.pitch) - 1, i = (int)(k % g.pitch) - OFFX;
    double* row = Kb + (long long)r * (bw + 1);
    const int ei[4] = {i - 1, i, i - 1, i}, ej[4] = {j - 1, j - 1, j, j}, eq[4] = {2, 3, 1, 0};
    for (int t = 0; t < 4; ++t) {
      if (ei[t] < 0 || ei[t] >= g.nx || ej[t] < 0 || ej[t] >= g.ny) continue;
      const long long ke = g.at(ei[t], ej[t]);
      double A[5][5] = {};
      A[0][0] = coef[ke];
      A[0][1] = A[1][0] = coef[s + ke];
      A[1][1] = coef[2 * s + ke];
      A[2][2] = coef[3 * s + ke];
      A[2][3] = A[3][2] = coef[4 * s + ke];
      A[3][3] = coef[5 * s + ke];
      A[0][2] = A[2][0] = coef[6 * s + ke];
      A[0][3] = A[3][0] = coef[7 * s + ke];
      A[1][2] = A[2][1] = coef[8 * s + ke];
      A[1][3] = A[3][1] = coef[9 * s + ke];
      A[4][4] = coef[10 * s + ke];
      A[1][4] = A[4][1] = coef[11 * s + ke];
      A[3][4] = A[4][3] = coef[12 * s + ke];
      // J column of this row's DOF.
      const int q = eq[t];
      const double s1 = (q == 1 || q == 2) ? 1.0 : -1.0, s2 = (q >= 2) ? 1.0 : -1.0;
      const double s3 = s1 * s2;  // s1 s2 = s3 (see elem_diag)
      double ja[5];
      if (c == 0) { ja[0] = s1; ja[1] = s3; ja[2] = 0; ja[3] = 0; ja[4] = s2; }
      else { ja[0] = 0; ja[1] = 0; ja[2] = s2; ja[3] = s3; ja[4] = s1; }
      double Aj[5];
      for (int m = 0; m < 5; ++m) {
        Aj[m] = 0.0;
        for (int l = 0; l < 5; ++l) Aj[m] += A[m][l] * ja[l];
      }
      // Element nodes: BL (ei, ej), BR, TR, TL.
      const int ni[4] = {ei[t], ei[t] + 1, ei[t] + 1, ei[t]}, nj[4] = {ej[t], ej[t], ej[t] + 1, ej[t] + 1};
      for (int m = 0; m < 4; ++m) {
        const double t1 = (m == 1 || m == 2) ? 1.0 : -1.0, t2 = (m >= 2) ? 1.0 : -1.0;
        const double t3 = t1 * t2;
        const long long kn = g.at(ni[m], nj[m]);
        const double ex = Aj[0] * t1 + Aj[1] * t3 + Aj[4] * t2;  // u_x column of node m
        const double ey = Aj[2] * t2 + Aj[3] * t3 + Aj[4] * t1;  // u_y column
        const int cx = dof_index[2 * kn], cy = dof_index[2 * kn + 1];
        if (cx >= 0 && cx <= r && r - cx <= bw) row[r - cx] += ex;
        if (cy >= 0 && cy <= r && r - cy <= bw) row[r - cy] += ey;
      }
    }
  }
}

// Right-looking band Cholesky (Alg. 3) with the next pivot taken off the
// critical path: one block of sixteen warps.  Step k scales column k by the
// pivot 1/L_kk computed in step k - 1, then updates the trailing triangle;
// warp 0 updates only the next diagonal entry (pair (0, 0)) and at once
// forms the next pivot (a reciprocal square root on the FP64 pipe), while
// warps 1-15 share the other pairs.  Two barriers per column.
constexpr int CHOL_NT = 512;

template <bool SMEM>
__global__ void __launch_bounds__(CHOL_NT)
    cholesky_band_kernel(int n, int bw, double* Bg, double* invL, double* Lsc, int* err) {
  extern __shared__ double dyn[];
  __shared__ double piv_s;
  const int W = bw + 1;
  double* B = SMEM ? dyn : Bg;
  short2* pairs = reinterpret_cast<short2*>(SMEM ? dyn + (size_t)n * W : dyn);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (SMEM)
    for (int t = tid; t < n * W; t += CHOL_NT) B[t] = Bg[t];
  for (int ii = tid; ii < bw; ii += CHOL_NT)
    for (int jj = 0; jj <= ii; ++jj) pairs[ii * (ii + 1) / 2 + jj] = make_short2((short)ii, (short)jj);
  __syncthreads();
  auto pivot = [&](int k) {
    double d = B[(size_t)k * W];
    if (!(d > 0.0) || !(d < 1.0e300)) {
      *err = 1;
      d = 1.0;
    }
    const double r = rsqrt(d);  // 1 / L_kk in one sequence (no separate division)
    B[(size_t)k * W] = d * r;
    piv_s = r;
    invL[k] = r;
  };
  if (tid == 0) pivot(0);
  __syncthreads();
  const int np_full = bw * (bw + 1) / 2;
  for (int k = 0; k < n; ++k) {
    const double piv = piv_s;
    const int last = min(n - 1, k + bw);
    const int m = last - k;
    for (int i = k + 1 + tid; i <= last; i += CHOL_NT) B[(size_t)i * W + (i - k)] *= piv;
    __syncthreads();
    if (warp == 0) {
      if (tid == 0 && m > 0) {
        const double l = B[(size_t)(k + 1) * W + 1];
        B[(size_t)(k + 1) * W] -= l * l;  // pair (0, 0): the next diagonal entry
        pivot(k + 1);
      }
    } else {
      const int np = m * (m + 1) / 2;
      for (int t = 1 + (tid - 32); t < np_full; t += CHOL_NT - 32) {
        const short2 pr = pairs[t];
        if (pr.x >= m) continue;  // rows beyond the matrix near the end
        const int i = k + 1 + pr.x, j = k + 1 + pr.y;
        B[(size_t)i * W + (i - j)] -= B[(size_t)i * W + (i - k)] * B[(size_t)j * W + (j - k)];
      }
      (void)np;
    }
    __syncthreads();
  }
  if (SMEM)
    for (int t = tid; t < n * W; t += CHOL_NT) Bg[t] = B[t];
  // The factor scaled by the pivots of its columns (Lsc[0 .. nW)) and of its
  // rows (Lsc[nW .. 2nW)), for the two substitutions of the inverse.
  for (int t = tid; t < n * W; t += CHOL_NT) {
    const int r = t / W, c = r - (t - r * W);
    const double v = B[t];
    Lsc[t] = c >= 0 ? v * invL[c] : 0.0;
    Lsc[(size_t)n * W + t] = v * invL[r];
  }
}

// K_0^-1 by columns: L y = e_j (forward), then L^T x = y (backward), column j
// stored in place in Kinv (row-major; K_0^-1 is symmetric, so this is also
// row j).  Eight threads share a column: thread t of the group takes the band
// terms d = t, t+8, ... of every row's dot product, the group adds its
// partial sums by shuffles, and every member then holds the new value.  Each
// thread keeps the last bw + 1 values of its column in a shared-memory ring
// (slot-major, so the 32 threads of a warp hit 32 distinct banks).  A warp
// carries four columns; one warp per block, so the blocks spread over the
// SMs, each with the factor broadcast from shared memory when it fits.
constexpr int INV_GROUP = 8;
constexpr int INV_COLS = 32 / INV_GROUP;

template <bool LSMEM>
__global__ void __launch_bounds__(32)
    inverse_cols_kernel(int n, int bw, const double* __restrict__ Lg, const double* __restrict__ invL,
                        double* __restrict__ Kinv) {
  extern __shared__ double dyn[];
  const int W = bw + 1;
  const int lane = threadIdx.x;
  const int t = lane % INV_GROUP;  // position inside the column group
  const double* L = Lg;
  double* win = dyn;
  if (LSMEM) {
    double* Ls = dyn;
    for (int q = lane; q < n * W; q += 32) Ls[q] = Lg[q];
    L = Ls;
    win = dyn + (size_t)n * W;
  }
  const int j0 = blockIdx.x * INV_COLS, j = j0 + lane / INV_GROUP;
  const bool active = j < n;
  for (int q = 0; q < W; ++q) win[q * 32 + lane] = 0.0;
  __syncwarp();
  // Forward substitution from row j0 (rows above j are zero for this column).
  int slot = j0 % W;
  for (int i = j0; i < n; ++i) {
    double a0 = 0.0, a1 = 0.0;
    const int dmax = min(bw, i);
    const double* Li = L + (size_t)i * W;
    int d = 1 + t;
    int sd = slot - d;
    if (sd < 0) sd += W;
    for (; d + INV_GROUP <= dmax; d += 2 * INV_GROUP) {
      const int sd2 = sd - INV_GROUP < 0 ? sd - INV_GROUP + W : sd - INV_GROUP;
      a0 += Li[d] * win[sd * 32 + lane];
      a1 += Li[d + INV_GROUP] * win[sd2 * 32 + lane];
      sd = sd2 - INV_GROUP < 0 ? sd2 - INV_GROUP + W : sd2 - INV_GROUP;
    }
    if (d <= dmax) a0 += Li[d] * win[sd * 32 + lane];
    double acc = a0 + a1;
#pragma unroll
    for (int o = 1; o < INV_GROUP; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const double y = ((i == j ? 1.0 : 0.0) - acc) * invL[i];
    win[slot * 32 + lane] = y;
    if (active && t == 0) Kinv[(size_t)i * n + j] = y;
    slot = slot + 1 == W ? 0 : slot + 1;
  }
  __syncwarp();
  for (int q = 0; q < W; ++q) win[q * 32 + lane] = 0.0;
  __syncwarp();
  // Backward substitution over all rows.
  slot = (n - 1) % W;
  for (int i = n - 1; i >= 0; --i) {
    const double yi = (i >= j0 && active) ? Kinv[(size_t)i * n + j] : 0.0;
    double a0 = 0.0, a1 = 0.0;
    const int dmax = min(bw, n - 1 - i);
    int d = 1 + t;
    int sd = slot + d;
    if (sd >= W) sd -= W;
    for (; d + INV_GROUP <= dmax; d += 2 * INV_GROUP) {
      const int sd2 = sd + INV_GROUP >= W ? sd + INV_GROUP - W : sd + INV_GROUP;
      a0 += L[(size_t)(i + d) * W + d] * win[sd * 32 + lane];
      a1 += L[(size_t)(i + d + INV_GROUP) * W + d + INV_GROUP] * win[sd2 * 32 + lane];
      sd = sd2 + INV_GROUP >= W ? sd2 + INV_GROUP - W : sd2 + INV_GROUP;
    }
    if (d <= dmax) a0 += L[(size_t)(i + d) * W + d] * win[sd * 32 + lane];
    double acc = a0 + a1;
#pragma unroll
    for (int o = 1; o < INV_GROUP; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const double x = (yi - acc) * invL[i];
    win[slot * 32 + lane] = x;
    __syncwarp();
    if (active && t == 0) Kinv[(size_t)i * n + j] = x;
    slot = slot == 0 ? W - 1 : slot - 1;
  }
}

// Element rows [j0, j1).  cp[p] = -penal E_p, so that a phase costs three
// FP64 operations (the kernel is bound by the FP64 pipe).
__global__ void sensitivity_kernel(int nelx, int nely, int j0, int j1, int n_phase,
                                   const double* __restrict__ x, PhaseTable cp, double penal,
                                   int ipenal, FineConst<double> kf, const double* __restrict__ u,
                                   double* __restrict__ dcdx, int accumulate) {
  const long long n = (long long)nelx * nely;
  const long long e1 = (long long)j1 * nelx;
  for (long long e = (long long)j0 * nelx + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < e1;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nelx), j = (int)(e / nelx);
    const long long n0 = (long long)j * (nelx + 1) + i, n3 = n0 + nelx + 1;
    const double2* u2 = reinterpret_cast<const double2*>(u);
    const double2 bl = u2[n0], br = u2[n0 + 1], tr = u2[n3 + 1], tl = u2[n3];
    const Strain<double> w = strain_coords<double>(bl, br, tr, tl);
    // u_e^T KE u_e in the strain basis (E = 1): kA (c1^2 + d2^2) + 2 kB c1 d2
    // + kC (c3^2 + d3^2) + kG s^2.
    const double a = fma(kf.kA, w.c1, (2.0 * kf.kB) * w.d2);
    const double b = fma(w.c3, w.c3, w.d3 * w.d3);
    const double we = fma(w.c1, a, fma(kf.kA * w.d2, w.d2, fma(kf.kC, b, (kf.kG * w.s) * w.s)));
    for (int p = 0; p < n_phase; ++p) {
      const long long k = (long long)p * n + e;
      const double xp = xpow(x[k], penal - 1.0, ipenal >= 1 ? ipenal - 1 : -1);
      const double g = (cp.E[p] * we) * xp;
      dcdx[k] = accumulate ? dcdx[k] + g : g;
    }
  }
}

// ---------------------------------------------------------------------------

static int blocks_for(long long n, int num_sms) {
  long long b = (n + 255) / 256;
  const long long cap = (long long)num_sms * 8;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

cudaError_t launch_modulus(const Grid& g, int n_phase, const double* x, PhaseTable ph, double penal,
                           int ipenal, double* E64, __nv_bfloat16* Ebf, double* Ek4,
                           FineConst<double> kf, cudaStream_t s, int num_sms, int j0, int j1) {
  if (j1 < 0) j1 = g.ny;
  if (j0 < 0 || j0 > j1 || j1 > g.ny) return cudaErrorInvalidValue;
  if (j0 == j1) return cudaSuccess;
  modulus_kernel<<<blocks_for((long long)g.nx * (j1 - j0), num_sms), 256, 0, s>>>(
      g, j0, j1, n_phase, x, ph, penal, ipenal, E64, Ebf, Ek4, kf);
  return cudaGetLastError();
}

cudaError_t launch_fine_invd(const Grid& g, const double* E64, double w_over_kdiag, double* invd1,
                             cudaStream_t s, int num_sms) {
  fine_invd_kernel<<<blocks_for((long long)(g.nx + 1) * (g.ny + 1), num_sms), 256, 0, s>>>(
      g, E64, w_over_kdiag, invd1);
  return cudaGetLastError();
}

cudaError_t launch_moments_from_fine(const Grid& gc, const Grid& gf, const double* E64,
                                     const __nv_bfloat16* Ebf, int rediscretize, double* mom,
                                     cudaStream_t s, int num_sms) {
  moments_from_fine_kernel<<<blocks_for((long long)gc.nx * gc.ny, num_sms), 256, 0, s>>>(
      gc, gf, E64, Ebf, rediscretize, mom);
  return cudaGetLastError();
}

cudaError_t launch_moments_from_coarse(const Grid& gc, const Grid& gf, const double* momf,
                                       int rediscretize, double* momc, cudaStream_t s, int num_sms) {
  moments_from_coarse_kernel<<<blocks_for((long long)gc.nx * gc.ny, num_sms), 256, 0, s>>>(
      gc, gf, momf, rediscretize, momc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coefs(const Grid& g, const double* mom, double nu, T* coef, cudaStream_t s,
                         int num_sms) {
  coefs_kernel<T><<<blocks_for((long long)g.nx * g.ny, num_sms), 256, 0, s>>>(g, mom, nu, coef);
  return cudaGetLastError();
}
template cudaError_t launch_coefs<double>(const Grid&, const double*, double, double*, cudaStream_t, int);
template cudaError_t launch_coefs<float>(const Grid&, const double*, double, float*, cudaStream_t, int);

template <typename T>
cudaError_t launch_coarse_invd(const Grid& g, const double* mom, double nu, double omega,
                               typename V2<T>::t* invd2, cudaStream_t s, int num_sms) {
  coarse_invd_kernel<T><<<blocks_for((long long)(g.nx + 1) * (g.ny + 1), num_sms), 256, 0, s>>>(
      g, mom, nu, omega, invd2);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_invd<double>(const Grid&, const double*, double, double, double2*,
                                                cudaStream_t, int);
template cudaError_t launch_coarse_invd<float>(const Grid&, const double*, double, double, float2*,
                                               cudaStream_t, int);

cudaError_t launch_kmom(const Grid& g, const double* mom, double nu, float* out, cudaStream_t s,
                        int num_sms) {
  kmom_kernel<<<blocks_for((long long)g.nx * g.ny, num_sms), 256, 0, s>>>(g, mom, nu, out);
  return cudaGetLastError();
}

cudaError_t launch_band_assemble(const Grid& g, const double* coef64, const int* dof_index, int n,
                                 int bw, double* Kb, cudaStream_t s) {
  band_assemble_kernel<<<(n + 127) / 128, 128, 0, s>>>(g, coef64, dof_index, n, bw, Kb);
  return cudaGetLastError();
}

static int max_dyn_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// K_0^-1 by columns with column-oriented (axpy) substitution: one warp per
// column j, four columns per block.  Forward, L y = e_j: at row k the warp
// has the running sum acc_k = sum_{m<k} L_km y_m ready, forms
// yh_k = delta_kj - acc_k = y_k L_kk (every lane the same value), and adds
// (L_rk / L_kk) yh_k to the sums of the next bw rows r, so the dependent chain
// of a step is one shuffle and one FP64 operation; y = yh / L_kk is formed in
// bulk after the pass.  The sums of a window of 32 NS rows live in
// registers: row r in lane r mod 32, slot (r / 32) mod NS, so a row's sum is
// broadcast by one shuffle and each step costs one FP64 operation per slot
// and lane (no reduction).  Backward, L^T x = y, runs the same way from the
// last row up with the factor scaled by its rows' pivots.  Column j of
// K_0^-1 is row j (symmetric).  Lsc holds the factor scaled by the pivots of
// its columns, then of its rows (cholesky_band_kernel); with LSMEM the block
// stages each in shared memory for its pass; each warp keeps its y in shared
// memory between the two passes.
constexpr int INVA_WARPS = 4;

template <bool LSMEM, int NS>
__global__ void __launch_bounds__(32 * INVA_WARPS)
    inverse_axpy_kernel(int n, int bw, const double* __restrict__ Lsc, const double* __restrict__ invL,
                        double* __restrict__ Kinv) {
  extern __shared__ double dyn[];
  constexpr int WIN = 32 * NS;
  const int W = bw + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* Lc = Lsc;                    // L_rk / L_kk
  const double* Lr = Lsc + (size_t)n * W;   // L_ir / L_ii
  const double* L = Lc;
  if (LSMEM) {
    for (int q = threadIdx.x; q < n * W; q += blockDim.x) dyn[q] = Lc[q];
    L = dyn;
  }
  double* ybuf = dyn + (LSMEM ? (size_t)n * W : 0) + (size_t)warp * n;
  __syncthreads();
  const int j = blockIdx.x * INVA_WARPS + warp;
  const bool active = j < n;  // the block's barriers below involve every warp
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  // Sum of row r, held by lane r % 32 in slot (r / 32) % NS, broadcast.
  auto take = [&](int r) -> double {
    const int sr = (r >> 5) & (NS - 1);
    double mine = acc[0];
#pragma unroll
    for (int s = 1; s < NS; ++s) mine = sr == s ? acc[s] : mine;
    const double v = __shfl_sync(0xffffffffu, mine, r & 31);
    if (lane == (r & 31)) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (sr == s) acc[s] = 0.0;  // the slot is reused for row r + WIN
    }
    return v;
  };
  if (active) {
    for (int k = j; k < n; ++k) {
      const double ak = take(k);
      const double yh = k == j ? 1.0 - ak : -ak;
      if (lane == 0) ybuf[k] = yh;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int o = (lane + 32 * s - (k + 1)) & (WIN - 1);  // row k + 1 + o
        const int r = k + 1 + o;
        if (o < bw && r < n) acc[s] = fma(L[(size_t)r * W + 1 + o], yh, acc[s]);
      }
    }
    __syncwarp();
    for (int k = j + lane; k < n; k += 32) ybuf[k] *= invL[k];
    __syncwarp();
  }
  if (LSMEM) {  // the factor scaled by its rows' pivots for the backward pass
    __syncthreads();
    for (int q = threadIdx.x; q < n * W; q += blockDim.x) dyn[q] = Lr[q];
    __syncthreads();
  } else {
    L = Lr;
  }
  if (!active) return;
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  double* row = Kinv + (size_t)j * n;
  for (int i = n - 1; i >= 0; --i) {
    const double yi = i >= j ? ybuf[i] : 0.0;
    const double ai = take(i);
    const double xh = yi - ai;  // x_i L_ii
    if (lane == 0) row[i] = xh;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int o = ((i - 1) - (lane + 32 * s)) & (WIN - 1);  // row i - 1 - o
      const int r = i - 1 - o;
      if (o < bw && r >= 0) acc[s] = fma(L[(size_t)i * W + 1 + o], xh, acc[s]);
    }
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) row[i] *= invL[i];
}

struct CholPlan {
  size_t pairs, band, win, ybuf;
  bool band_smem, inv_smem, axpy_smem;
  int slots;  // register slots of the axpy inverse (0: use inverse_cols_kernel)
};

static CholPlan chol_plan(int n, int bw) {
  CholPlan p;
  const int W = bw + 1;
  p.pairs = sizeof(short2) * (size_t)bw * (bw + 1) / 2 + 16;
  p.band = sizeof(double) * (size_t)n * W;
  p.win = sizeof(double) * (size_t)W * 32;
  p.ybuf = sizeof(double) * (size_t)n * INVA_WARPS;
  const int cap = max_dyn_smem();
  p.band_smem = p.band + p.pairs <= (size_t)cap;
  p.inv_smem = p.band + p.win <= (size_t)cap;
  p.axpy_smem = p.band + p.ybuf <= (size_t)cap;
  p.slots = bw < 64 ? 2 : (bw < 128 ? 4 : 0);
  if (p.ybuf > (size_t)cap) p.slots = 0;
  return p;
}

template <bool LSMEM, int NS> static cudaError_t set_axpy_smem(size_t bytes) {
  return raise_max_dynamic_smem((const void*)inverse_axpy_kernel<LSMEM, NS>, bytes);
}

cudaError_t prepare_cholesky_inverse(int n, int bw) {
  const CholPlan pl = chol_plan(n, bw);
  cudaError_t e = cudaSuccess;
  if (pl.band_smem)
    e = raise_max_dynamic_smem((const void*)cholesky_band_kernel<true>, pl.band + pl.pairs);
  else
    e = raise_max_dynamic_smem((const void*)cholesky_band_kernel<false>, pl.pairs);
  if (e != cudaSuccess) return e;
  if (pl.slots == 2) {
    return pl.axpy_smem ? set_axpy_smem<true, 2>(pl.band + pl.ybuf) : set_axpy_smem<false, 2>(pl.ybuf);
  }
  if (pl.slots == 4) {
    return pl.axpy_smem ? set_axpy_smem<true, 4>(pl.band + pl.ybuf) : set_axpy_smem<false, 4>(pl.ybuf);
  }
  if (pl.inv_smem)
    e = raise_max_dynamic_smem((const void*)inverse_cols_kernel<true>, pl.band + pl.win);
  else
    e = raise_max_dynamic_smem((const void*)inverse_cols_kernel<false>, pl.win);
  return e;
}

cudaError_t launch_cholesky_inverse(int n, int bw, double* Kb, double* invL, double* Lsc, double* Kinv,
                                    int* err_flag, cudaStream_t s, int num_sms) {
  (void)num_sms;
  const CholPlan pl = chol_plan(n, bw);
  if (pl.band_smem)
    cholesky_band_kernel<true><<<1, CHOL_NT, pl.band + pl.pairs, s>>>(n, bw, Kb, invL, Lsc, err_flag);
  else
    cholesky_band_kernel<false><<<1, CHOL_NT, pl.pairs, s>>>(n, bw, Kb, invL, Lsc, err_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (pl.slots) {
    const int ab = (n + INVA_WARPS - 1) / INVA_WARPS;
    const size_t sm = (pl.axpy_smem ? pl.band : 0) + pl.ybuf;
    if (pl.slots == 2) {
      if (pl.axpy_smem) inverse_axpy_kernel<true, 2><<<ab, 32 * INVA_WARPS, sm, s>>>(n, bw, Lsc, invL, Kinv);
      else inverse_axpy_kernel<false, 2><<<ab, 32 * INVA_WARPS, sm, s>>>(n, bw, Lsc, invL, Kinv);
    } else {
      if (pl.axpy_smem) inverse_axpy_kernel<true, 4><<<ab, 32 * INVA_WARPS, sm, s>>>(n, bw, Lsc, invL, Kinv);
      else inverse_axpy_kernel<false, 4><<<ab, 32 * INVA_WARPS, sm, s>>>(n, bw, Lsc, invL, Kinv);
    }
    return cudaGetLastError();
  }
  const int blocks = (n + INV_COLS - 1) / INV_COLS;
  if (pl.inv_smem)
    inverse_cols_kernel<true><<<blocks, 32, pl.band + pl.win, s>>>(n, bw, Kb, invL, Kinv);
  else
    inverse_cols_kernel<false><<<blocks, 32, pl.win, s>>>(n, bw, Kb, invL, Kinv);
  return cudaGetLastError();
}

cudaError_t launch_sensitivity(int nelx, int nely, int n_phase, const double* x, PhaseTable ph,
                               double penal, int ipenal, FineConst<double> kf, const double* u,
                               double* dcdx, int accumulate, cudaStream_t s, int num_sms, int j0,
                               int j1) {
  if (j1 < 0) j1 = nely;
  if (j0 < 0 || j0 > j1 || j1 > nely) return cudaErrorInvalidValue;
  if (j0 == j1) return cudaSuccess;
  PhaseTable cp{};
  for (int p = 0; p < n_phase && p < 16; ++p) cp.E[p] = -penal * ph.E[p];
  sensitivity_kernel<<<blocks_for((long long)nelx * (j1 - j0), num_sms), 256, 0, s>>>(
      nelx, nely, j0, j1, n_phase, x, cp, penal, ipenal, kf, u, dcdx, accumulate);
  return cudaGetLastError();
}

}  // namespace mto
