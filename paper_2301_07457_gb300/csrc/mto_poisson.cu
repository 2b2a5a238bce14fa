// Scalar Poisson pCGMG (Sec. 5.1): -Laplace(u) = f on an nelx x nely mesh of
// unit Q4 elements, u = 0 on the four edges, solved by PCG (Alg. 2)
// preconditioned by one V-cycle (Alg. 1) with damped-Jacobi smoothing
// (Sec. 2.3), bilinear transfers and a dense inverse on the coarsest grid
// (factored by Alg. 3).
//
// The assembled constant-coefficient Q4 Laplacian is the 9-point stencil
// (K u)(n) = (8 u_n - sum of the 8 neighbours) / 3, its diagonal 8/3.  The
// Galerkin coarse operator P^T K P with bilinear P is the same stencil on
// every grid (the 2-D element matrix does not depend on the element size),
// so no coarse operator is stored.
//
// Execution: the whole solve is ONE kernel launch.  Each right-hand side is
// solved by one thread-block cluster of C CTAs (C = 1 for small meshes, up to
// 16): the CTAs own blocks of node rows of every large level and separate
// dependent phases with the hardware cluster barrier; scalar reductions are
// all-gathered through distributed shared memory and summed in rank order,
// so every CTA holds the same scalars and takes the same branches.  Levels
// with at most LOCAL_MAX_NODES (256) interior nodes (and the coarsest solve)
// run inside CTA 0 alone with block barriers.  All vectors live in global memory
// (a few MB: L2-resident).  There is no spin-wait: every barrier is a
// hardware barrier of the block or the cluster.
#include <cooperative_groups.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mto_ctx.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int PNT = 256;                // threads per CTA (255 registers each)
constexpr int PWARPS = PNT / 32;
constexpr int PMAXC = 16;               // CTAs per cluster (non-portable above 8)
constexpr int PMAXL = 16;               // grids
constexpr int LOCAL_MAX_NODES = 256;    // interior nodes of a level run by CTA 0 alone
constexpr int PMAX_COARSE = 1024;       // interior nodes of the coarsest grid (dense inverse)
constexpr int PMAX_RHS = 64;

enum { PMODE_SOLVE = 0, PMODE_PRECOND = 1, PMODE_APPLY = 2 };
enum { PST_RUNNING = 0, PST_CONVERGED = 1, PST_MAXIT = 2, PST_BREAKDOWN = 3 };

struct PLevel {
  int nx, ny;       // elements; nodes (nx + 1) x (ny + 1), row pitch nx + 1
  void* z[2];       // iterates (ping-pong) in the V-cycle's type; boundary entries stay zero
  void* b;          // right-hand side (coarse levels), same type
};

struct PStats {
  int iters, status;
  double rr, ff, rr_true;
};

struct PDesc {
  int L, fl;                 // finest level; levels 0..fl run on CTA 0 alone
  int mode, nu1, nu2, max_it, flexible;
  double tol2, wd;           // tol^2, omega / D = 3 omega / 8
  int n0;                    // interior nodes of the coarsest grid
  const double* Kinv;        // n0 x n0, row-major
  const double* f;           // finest right-hand side / input vector (nodal layout)
  double* x;                 // finest iterate (solve), output (precond / apply)
  double *r, *p, *q;         // finest CG vectors
  PStats* stats;
  PLevel lv[PMAXL];
};

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
// Work split of a phase: this CTA's block of interior node rows [j0, j1) of a
// level with ny elements in y, and its rank / size (1 for CTA-local phases).
struct Part {
  int rank, size;
};

__device__ __forceinline__ void rows_of(int ny, Part pt, int& j0, int& j1) {
  const int rows = ny - 1;
  const int per = (rows + pt.size - 1) / pt.size;
  j0 = 1 + pt.rank * per;
  j1 = min(ny, j0 + per);
}

// For every interior node of this CTA's rows: v = ld(i, j, k), then st(k, v).
// Each thread takes NB nodes at a time and evaluates ld (loads and
// arithmetic, no stores) for all of them before the first st, so that the
// loads of the NB nodes are in flight together: a phase then costs about
// nodes / (NB * threads) memory round trips instead of nodes / threads.
template <int NB, typename Ld, typename St>
__device__ __forceinline__ void for_nodes_nb(int nx, int ny, Part pt, Ld ld, St st) {
  int j0, j1;
  rows_of(ny, pt, j0, j1);
  const int w = nx - 1;
  const int count = (j1 - j0) * w;
  for (int t0 = threadIdx.x; t0 < count; t0 += NB * PNT) {
    decltype(ld(0, 0, 0)) v[NB];
    int ks[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int t = t0 + u * PNT;
      ks[u] = -1;
      if (t < count) {
        const int j = j0 + t / w;
        const int i = 1 + t % w;
        ks[u] = j * (nx + 1) + i;
        v[u] = ld(i, j, ks[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u)
      if (ks[u] >= 0) st(ks[u], v[u]);
  }
}

// Calls fn(i, j, k) for every interior node of this CTA's rows.
template <typename F> __device__ __forceinline__ void for_nodes(int nx, int ny, Part pt, F fn) {
  int j0, j1;
  rows_of(ny, pt, j0, j1);
  const int w = nx - 1;
  const int count = (j1 - j0) * w;
  for (int t = threadIdx.x; t < count; t += PNT) {
    const int j = j0 + t / w;
    const int i = 1 + t % w;
    fn(i, j, j * (nx + 1) + i);
  }
}

}  // namespace

namespace {

struct PShared {
  double red[5][PMAXC];   // all-gathered partial sums, one row per reduction slot
  double warp[2][PWARPS];
};

// Reduction slots (each used once per PCG iteration, so that consecutive
// uses of a slot are separated by several barriers).
enum { SLOT_RHO = 0, SLOT_PQ = 1, SLOT_RR = 2, SLOT_FF = 3, SLOT_TRUE = 3, SLOT_ZQ = 4 };

// The 9-point stencil on a vector of type T, evaluated in float64.
template <typename T> __device__ __forceinline__ double apply_k64(const T* z, int k, int pitch) {
  auto v = [&](int o) { return (double)z[k + o]; };
  const double s = (v(-pitch - 1) + v(-pitch) + v(-pitch + 1)) + (v(-1) + v(1)) +
                   (v(pitch - 1) + v(pitch) + v(pitch + 1));
  return (8.0 * v(0) - s) * (1.0 / 3.0);
}

template <typename T> __device__ __forceinline__ T nbsum_t(const T* z, int k, int pitch) {
  return (z[k - pitch - 1] + z[k - pitch] + z[k - pitch + 1]) + (z[k - 1] + z[k + 1]) +
         (z[k + pitch - 1] + z[k + pitch] + z[k + pitch + 1]);
}

template <typename T> __device__ __forceinline__ T prolong_t(const T* zc, int pc, int i, int j) {
  const int I = i >> 1, J = j >> 1;
  const int k = J * pc + I;
  const T h = T(0.5), qt = T(0.25);
  if (!(j & 1)) return (i & 1) ? h * (zc[k] + zc[k + 1]) : zc[k];
  if (!(i & 1)) return h * (zc[k] + zc[k + pc]);
  return qt * ((zc[k] + zc[k + 1]) + (zc[k + pc] + zc[k + pc + 1]));
}

// The V-cycle runs in VT (double, or float for the mixed precision); the
// CG vectors, dot products and the stopping test are float64 in both.
template <typename VT> struct Solver {
  const PDesc& d;
  PShared& sh;
  int rank, C;
  cg::cluster_group cl;

  __device__ Part part(bool cluster) const { return cluster ? Part{rank, C} : Part{0, 1}; }
  __device__ void sync(bool cluster) {
    if (cluster) cl.sync();
    else __syncthreads();
  }
  __device__ VT* Z(int l, int i) const { return static_cast<VT*>(d.lv[l].z[i]); }
  __device__ VT* B(int l) const { return static_cast<VT*>(d.lv[l].b); }
  // Iterate buffers: the pre-smoothed iterate and the final one of level l.
  __device__ int pre_buf() const { return (d.nu1 - 1) & 1; }
  __device__ int final_buf(int l) const { return l == 0 ? 0 : (d.nu1 - 1 + d.nu2) & 1; }

  // Sum of a (and b) over the cluster, in rank order; every thread of every
  // CTA gets the same result.  Includes the phase barrier.
  __device__ void allreduce(double& a, double& b, int slot_a, int slot_b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      sh.warp[0][w] = a;
      sh.warp[1][w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sa = 0.0, sb = 0.0;
      for (int i = 0; i < PWARPS; ++i) {
        sa += sh.warp[0][i];
        sb += sh.warp[1][i];
      }
      if (C > 1) {
        for (int dst = 0; dst < C; ++dst) {
          cl.map_shared_rank(&sh.red[slot_a][0], dst)[rank] = sa;
          if (slot_b >= 0) cl.map_shared_rank(&sh.red[slot_b][0], dst)[rank] = sb;
        }
      } else {
        sh.red[slot_a][0] = sa;
        if (slot_b >= 0) sh.red[slot_b][0] = sb;
      }
    }
    sync(C > 1);
    a = 0.0;
    b = 0.0;
    for (int i = 0; i < C; ++i) {
      a += sh.red[slot_a][i];
      if (slot_b >= 0) b += sh.red[slot_b][i];
    }
  }
  __device__ double allreduce1(double a, int slot) {
    double b = 0.0;
    allreduce(a, b, slot, -1);
    return a;
  }

  // dst = src + (omega / D)(b - K src) on level l, in VT:
  // (1 - 8 w/(3D)) z + w/D b + w/(3D) s with s the sum of the 8 neighbours
  // (7 additions, one multiplication, two FMAs).  With dotv (and dotq) the
  // float64 sums dst . dotv (dst . dotq) over this CTA's nodes are added to
  // acc (accq).
  template <typename BT>
  __device__ void sweep(int l, const VT* src, VT* dst, const BT* b, bool cluster, const double* dotv,
                        const double* dotq, double& acc, double& accq) {
    const PLevel& lv = d.lv[l];
    const int pitch = lv.nx + 1;
    const VT wd = VT(d.wd), cz = VT(1.0 - 8.0 * d.wd / 3.0), cs = VT(d.wd / 3.0);
    // Nodes in flight per thread: as many as the 255-register budget holds.
    constexpr int NB = sizeof(VT) == 8 ? 4 : 8;
    for_nodes_nb<NB>(
        lv.nx, lv.ny, part(cluster),
        [&](int, int, int k) {
          return fma(cz, src[k], fma(wd, VT(b[k]), cs * nbsum_t(src, k, pitch)));
        },
        [&](int k, VT v) {
          dst[k] = v;
          if (dotv) acc = fma((double)v, dotv[k], acc);
          if (dotq) accq = fma((double)v, dotq[k], accq);
        });
  }

  // The prolongation and correction z += P zc of level l, in place
  // (pointwise: each node reads itself and at most four coarse nodes).
  __device__ void prolong_add(int l, VT* z, const VT* zc, bool cluster) {
    const PLevel& lv = d.lv[l];
    const int pc = d.lv[l - 1].nx + 1;
    for_nodes_nb<4>(
        lv.nx, lv.ny, part(cluster),
        [&](int i, int j, int k) { return z[k] + prolong_t(zc, pc, i, j); },
        [&](int k, VT v) { z[k] = v; });
  }

  // The residual res = b - K zpre of level l (interior nodes), in VT.
  template <typename BT>
  __device__ void residual(int l, const VT* zpre, const BT* b, VT* res, bool cluster) {
    const PLevel& lv = d.lv[l];
    const int pitch = lv.nx + 1;
    const VT third = VT(1.0 / 3.0);
    for_nodes_nb<4>(
        lv.nx, lv.ny, part(cluster),
        [&](int, int, int k) { return VT(b[k]) - (VT(8) * zpre[k] - nbsum_t(zpre, k, pitch)) * third; },
        [&](int k, VT v) { res[k] = v; });
  }

  // Full-weighting restriction R = P^T of the fine residual res into the
  // right-hand side of level l - 1, and that level's first smoothing step
  // from zero, z = (omega / D) b (pointwise), unless it is the coarsest grid.
  __device__ void restrict_to(int l, const VT* res, bool cluster) {
    const int pf = d.lv[l].nx + 1;
    const PLevel& c = d.lv[l - 1];
    VT* bc = B(l - 1);
    VT* z0 = Z(l - 1, 0);
    const VT wd = VT(d.wd), h = VT(0.5), qt = VT(0.25);
    const bool first = l - 1 >= 1;
    for_nodes_nb<4>(
        c.nx, c.ny, part(cluster),
        [&](int I, int J, int) {
          const int k = 2 * J * pf + 2 * I;
          return res[k] + h * ((res[k - 1] + res[k + 1]) + (res[k - pf] + res[k + pf])) +
                 qt * ((res[k - pf - 1] + res[k - pf + 1]) + (res[k + pf - 1] + res[k + pf + 1]));
        },
        [&](int kc, VT v) {
          bc[kc] = v;
          if (first) z0[kc] = wd * v;
        });
  }

  // Float32 V-cycle only: the residual formed on the fly at the nine fine
  // nodes of each coarse node inside the restriction, and the prolongation
  // formed on the fly at the node and its neighbours inside the first
  // post-smoothing sweep.  The recomputation costs float32 operations, which
  // are cheap here, and saves two barriers per grid.
  template <typename BT>
  __device__ void restrict_fused(int l, const VT* zpre, const BT* b, bool cluster) {
    const int pf = d.lv[l].nx + 1;
    const PLevel& c = d.lv[l - 1];
    VT* bc = B(l - 1);
    VT* z0 = Z(l - 1, 0);
    const VT wd = VT(d.wd), h = VT(0.5), qt = VT(0.25), third = VT(1.0 / 3.0);
    const bool first = l - 1 >= 1;
    for_nodes_nb<2>(
        c.nx, c.ny, part(cluster),
        [&](int I, int J, int) {
          const int k = 2 * J * pf + 2 * I;
          auto res = [&](int kk) { return VT(b[kk]) - (VT(8) * zpre[kk] - nbsum_t(zpre, kk, pf)) * third; };
          return res(k) + h * ((res(k - 1) + res(k + 1)) + (res(k - pf) + res(k + pf))) +
                 qt * ((res(k - pf - 1) + res(k - pf + 1)) + (res(k + pf - 1) + res(k + pf + 1)));
        },
        [&](int kc, VT v) {
          bc[kc] = v;
          if (first) z0[kc] = wd * v;
        });
  }

  template <typename BT>
  __device__ void prolong_sweep(int l, const VT* zpre, const VT* zc, VT* dst, const BT* b, bool cluster,
                                const double* dotv, const double* dotq, double& acc, double& accq) {
    const PLevel& lv = d.lv[l];
    const int pitch = lv.nx + 1, pc = d.lv[l - 1].nx + 1;
    const VT wd = VT(d.wd), cz = VT(1.0 - 8.0 * d.wd / 3.0), cs = VT(d.wd / 3.0);
    for_nodes_nb<2>(
        lv.nx, lv.ny, part(cluster),
        [&](int i, int j, int k) {
          auto zf = [&](int di, int dj) {
            return zpre[k + dj * pitch + di] + prolong_t(zc, pc, i + di, j + dj);
          };
          const VT s = (zf(-1, -1) + zf(0, -1) + zf(1, -1)) + (zf(-1, 0) + zf(1, 0)) +
                       (zf(-1, 1) + zf(0, 1) + zf(1, 1));
          return fma(cz, zf(0, 0), fma(wd, VT(b[k]), cs * s));
        },
        [&](int k, VT v) {
          dst[k] = v;
          if (dotv) acc = fma((double)v, dotv[k], acc);
          if (dotq) accq = fma((double)v, dotq[k], accq);
        });
  }

  // Coarsest grid: z = K_0^-1 b (float64 dense inverse, one warp per row).
  __device__ void coarsest() {
    const PLevel& c = d.lv[0];
    const VT* b0 = B(0);
    VT* z0 = Z(0, 0);
    const int n = d.n0, w = c.nx - 1, pitch = c.nx + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int a = warp; a < n; a += PWARPS) {
      double s = 0.0;
      for (int bb = lane; bb < n; bb += 32)
        s = fma(d.Kinv[(size_t)a * n + bb], (double)b0[(1 + bb / w) * pitch + 1 + bb % w], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) z0[(1 + a / w) * pitch + 1 + a % w] = VT(s);
    }
  }

  // Pre-smoothing (the first step from zero is already in z[0]), the
  // residual (into the free buffer of the pair) and its restriction, level l.
  template <typename BT> __device__ void descend(int l, const BT* b, bool cluster) {
    int cur = 0;
    double u = 0.0, v = 0.0;
    for (int s = 1; s < d.nu1; ++s) {
      sweep(l, Z(l, cur), Z(l, cur ^ 1), b, cluster, nullptr, nullptr, u, v);
      cur ^= 1;
      sync(cluster);
    }
    if constexpr (sizeof(VT) == 4) {
      restrict_fused(l, Z(l, cur), b, cluster);
    } else {
      residual(l, Z(l, cur), b, Z(l, cur ^ 1), cluster);
      sync(cluster);
      restrict_to(l, Z(l, cur ^ 1), cluster);
    }
    sync(cluster);
  }

  // Prolongation and correction, then post-smoothing of level l.  With dotv,
  // the last sweep also forms the partial sums z . dotv (and z . dotq) and
  // its barrier is left to the reduction that follows.
  template <typename BT>
  __device__ void ascend(int l, const BT* b, bool cluster, const double* dotv, const double* dotq,
                         double& acc, double& accq) {
    int cur = pre_buf();
    int s0 = 0;
    if constexpr (sizeof(VT) == 4) {
      const bool last = d.nu2 == 1;
      prolong_sweep(l, Z(l, cur), Z(l - 1, final_buf(l - 1)), Z(l, cur ^ 1), b, cluster,
                    last ? dotv : nullptr, last ? dotq : nullptr, acc, accq);
      cur ^= 1;
      s0 = 1;
    } else {
      prolong_add(l, Z(l, cur), Z(l - 1, final_buf(l - 1)), cluster);
    }
    for (int s = s0; s < d.nu2; ++s) {
      sync(cluster);
      const bool last = s == d.nu2 - 1;
      sweep(l, Z(l, cur), Z(l, cur ^ 1), b, cluster, last ? dotv : nullptr, last ? dotq : nullptr, acc,
            accq);
      cur ^= 1;
    }
    if (!dotv) sync(cluster);
  }

  // One V-cycle (Alg. 1 with gamma = 1) for the finest right-hand side bL
  // (float64), whose first smoothing step is already in Z(L, 0).  With dotv
  // (dotq), this CTA's part of z . dotv (z . dotq) is added to acc (accq);
  // the caller reduces them.
  __device__ void vcycle(const double* bL, const double* dotv, const double* dotq, double& acc,
                         double& accq) {
    const int L = d.L;
    const int top_local = C > 1 ? d.fl : L;
    for (int l = L; l > top_local; --l) {
      if (l == L) descend(l, bL, true);
      else descend(l, static_cast<const VT*>(B(l)), true);
    }
    if (C == 1 || rank == 0) {
      for (int l = top_local; l >= 1; --l) {
        if (l == L) descend(l, bL, false);
        else descend(l, static_cast<const VT*>(B(l)), false);
      }
      coarsest();
      __syncthreads();
      for (int l = 1; l <= top_local; ++l) {
        if (l == L) ascend(l, bL, false, dotv, dotq, acc, accq);
        else ascend(l, static_cast<const VT*>(B(l)), false, nullptr, nullptr, acc, accq);
      }
    }
    if (C > 1) cl.sync();
    for (int l = top_local + 1; l <= L; ++l) {
      if (l == L) ascend(l, bL, true, dotv, dotq, acc, accq);
      else ascend(l, static_cast<const VT*>(B(l)), true, nullptr, nullptr, acc, accq);
    }
  }

  // ------------------------------------------------------------------------
  // Alg. 2 with the V-cycle above as preconditioner; stop when
  // ||r|| <= tol ||f|| (tested before the preconditioner).  beta is
  // Fletcher-Reeves (float64 V-cycle) or the flexible form
  // z_i . (r_i - r_{i-1}) / rho_{i-1} = -alpha_{i-1} z_i . q_{i-1} / rho_{i-1}
  // (float32 V-cycle), with z . q formed in the last smoothing sweep.
  // q = K p is formed as K z + beta q (K is linear, evaluated in float64), so
  // that the phase needs z at the neighbours (complete after the V-cycle's
  // last barrier) but p only at the node itself.
  // ------------------------------------------------------------------------
  __device__ void solve() {
    const PLevel& F = d.lv[d.L];
    const int nx = F.nx, ny = F.ny, pitch = nx + 1;
    const bool cl_on = C > 1;
    const Part pt = part(cl_on);
    double* x = d.x;
    double *r = d.r, *p = d.p, *q = d.q;
    const double* f = d.f;
    VT* z0 = Z(d.L, 0);
    const double wd = d.wd;
    // Warm start: the iterate is zero on the boundary.
    if (rank == 0) {
      for (int t = threadIdx.x; t < nx + 1; t += PNT) {
        x[t] = 0.0;
        x[ny * pitch + t] = 0.0;
      }
      for (int t = threadIdx.x; t < ny + 1; t += PNT) {
        x[t * pitch] = 0.0;
        x[t * pitch + nx] = 0.0;
      }
    }
    sync(cl_on);
    double rr = 0.0, ff = 0.0;
    for_nodes(nx, ny, pt, [&](int, int, int k) {
      const double rk = f[k] - apply_k64(x, k, pitch);
      r[k] = rk;
      z0[k] = VT(wd * rk);
      rr = fma(rk, rk, rr);
      ff = fma(f[k], f[k], ff);
    });
    allreduce(rr, ff, SLOT_RR, SLOT_FF);
    int it = 0, status = PST_RUNNING;
    double rho_old = 1.0, alpha_old = 0.0;
    const VT* z = Z(d.L, final_buf(d.L));
    constexpr int NBC = sizeof(VT) == 8 ? 4 : 8;  // nodes in flight per thread (registers)
    for (;;) {
      if (!isfinite(rr)) {
        status = PST_BREAKDOWN;
        break;
      }
      if (rr <= d.tol2 * ff) {
        status = PST_CONVERGED;
        break;
      }
      if (it >= d.max_it) {
        status = PST_MAXIT;
        break;
      }
      // The flexible form belongs to the float32 V-cycle (compiled out of
      // the float64 one).
      constexpr bool FLEX = sizeof(VT) == 4;
      const bool flex = FLEX && d.flexible && it > 0;
      double rho = 0.0, zq = 0.0;
      if constexpr (FLEX) {
        vcycle(r, r, flex ? q : nullptr, rho, zq);
        if (flex) allreduce(rho, zq, SLOT_RHO, SLOT_ZQ);
        else rho = allreduce1(rho, SLOT_RHO);
      } else {
        vcycle(r, r, nullptr, rho, zq);
        rho = allreduce1(rho, SLOT_RHO);
      }
      if (!(rho > 0.0) || !isfinite(rho)) {
        status = PST_BREAKDOWN;
        break;
      }
      const double beta = it == 0 ? 0.0 : (flex ? -alpha_old * zq / rho_old : rho / rho_old);
      double pq = 0.0;
      for_nodes_nb<NBC>(
          nx, ny, pt,
          [&](int, int, int k) {
            const double kz = apply_k64(z, k, pitch);
            const double zk = (double)z[k];
            const double pk = it == 0 ? zk : fma(beta, p[k], zk);
            const double qk = it == 0 ? kz : fma(beta, q[k], kz);
            return double2{pk, qk};
          },
          [&](int k, double2 v) {
            p[k] = v.x;
            q[k] = v.y;
            pq = fma(v.x, v.y, pq);
          });
      pq = allreduce1(pq, SLOT_PQ);
      if (!(pq > 0.0) || !isfinite(pq)) {
        status = PST_BREAKDOWN;
        break;
      }
      const double alpha = rho / pq;
      double rn = 0.0;
      for_nodes_nb<NBC>(
          nx, ny, pt,
          [&](int, int, int k) { return double2{fma(alpha, p[k], x[k]), fma(-alpha, q[k], r[k])}; },
          [&](int k, double2 v) {
            x[k] = v.x;
            r[k] = v.y;
            z0[k] = VT(wd * v.y);  // the next V-cycle's first smoothing step from zero
            rn = fma(v.y, v.y, rn);
          });
      rr = allreduce1(rn, SLOT_RR);
      rho_old = rho;
      alpha_old = alpha;
      ++it;
    }
    // True residual of the returned iterate.
    double rt = 0.0;
    for_nodes(nx, ny, pt, [&](int, int, int k) {
      const double rk = f[k] - apply_k64(x, k, pitch);
      rt = fma(rk, rk, rt);
    });
    rt = allreduce1(rt, SLOT_TRUE);
    if (rank == 0 && threadIdx.x == 0) {
      d.stats->iters = it;
      d.stats->status = status;
      d.stats->rr = rr;
      d.stats->ff = ff;
      d.stats->rr_true = rt;
    }
  }

  // z = one V-cycle applied to the input vector (the preconditioner alone).
  __device__ void precondition() {
    const PLevel& F = d.lv[d.L];
    const bool cl_on = C > 1;
    const double wd = d.wd;
    const double* v = d.f;
    VT* z0 = Z(d.L, 0);
    for_nodes(F.nx, F.ny, part(cl_on), [&](int, int, int k) { z0[k] = VT(wd * v[k]); });
    sync(cl_on);
    double u = 0.0, w = 0.0;
    vcycle(v, nullptr, nullptr, u, w);
    const VT* z = Z(d.L, final_buf(d.L));
    const int n = (F.nx + 1) * (F.ny + 1);
    const int per = (n + C - 1) / C;
    const int a = rank * per, e = min(n, a + per);
    for (int k = a + threadIdx.x; k < e; k += PNT) d.x[k] = (double)z[k];  // zero on the boundary
    sync(cl_on);
  }

  // y = K v (float64) with v read as zero on the boundary.
  __device__ void apply() {
    const PLevel& F = d.lv[d.L];
    const int nx = F.nx, ny = F.ny, pitch = nx + 1;
    const double* v = d.f;
    double* y = d.x;
    for_nodes(nx, ny, part(C > 1), [&](int i, int j, int k) {
      auto vv = [&](int di, int dj) {
        const int ii = i + di, jj = j + dj;
        return (ii == 0 || ii == nx || jj == 0 || jj == ny) ? 0.0 : v[k + dj * pitch + di];
      };
      const double s = (vv(-1, -1) + vv(0, -1) + vv(1, -1)) + (vv(-1, 0) + vv(1, 0)) +
                       (vv(-1, 1) + vv(0, 1) + vv(1, 1));
      y[k] = (8.0 * v[k] - s) * (1.0 / 3.0);
    });
    if (rank == 0) {
      for (int t = threadIdx.x; t < nx + 1; t += PNT) {
        y[t] = 0.0;
        y[ny * pitch + t] = 0.0;
      }
      for (int t = threadIdx.x; t < ny + 1; t += PNT) {
        y[t * pitch] = 0.0;
        y[t * pitch + nx] = 0.0;
      }
    }
    sync(C > 1);
  }
};

// One cluster of C CTAs per descriptor (right-hand side); VT is the V-cycle's
// value type.
template <typename VT>
__global__ void __launch_bounds__(PNT, 1) poisson_cluster_kernel(const PDesc* __restrict__ descs, int C) {
  __shared__ PDesc sd;
  __shared__ PShared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const PDesc* src = descs + blockIdx.x / C;
  {
    const int* s = reinterpret_cast<const int*>(src);
    int* t = reinterpret_cast<int*>(&sd);
    for (int i = threadIdx.x; i < (int)(sizeof(PDesc) / sizeof(int)); i += PNT) t[i] = s[i];
  }
  __syncthreads();
  Solver<VT> s{sd, sh, rank, C, cl};
  if (sd.mode == PMODE_SOLVE) s.solve();
  else if (sd.mode == PMODE_PRECOND) s.precondition();
  else s.apply();
}

// Coarsest grid (one CTA): band Cholesky of K_0 (Alg. 3, right-looking, in
// the lower band Ab[i * (bw + 1) + i - j]), then K_0^-1 column by column by
// forward and back substitution.  err is set when a pivot is not positive.
__global__ void __launch_bounds__(PNT) poisson_coarsest_kernel(int nx0, int ny0, double* Ab,
                                                               double* Kinv, int* err) {
  const int w = nx0 - 1, n = w * (ny0 - 1), bw = w + 1, ld = bw + 1;
  for (int t = threadIdx.x; t < n * ld; t += PNT) {
    const int i = t / ld, dd = t % ld, j = i - dd;
    double v = 0.0;
    if (j >= 0) {
      const int dx = i % w - j % w, dy = i / w - j / w;
      if (dd == 0) v = 8.0 / 3.0;
      else if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) v = -1.0 / 3.0;
    }
    Ab[t] = v;
  }
  __syncthreads();
  __shared__ double piv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double a = Ab[(size_t)k * ld];
      if (!(a > 0.0)) *err = 1;
      piv = sqrt(a > 0.0 ? a : 1.0);
      Ab[(size_t)k * ld] = piv;
    }
    __syncthreads();
    const int m = min(n - 1, k + bw);
    for (int i = k + 1 + threadIdx.x; i <= m; i += PNT) Ab[(size_t)i * ld + (i - k)] /= piv;
    __syncthreads();
    const int cnt = m - k;
    for (int t = threadIdx.x; t < cnt * cnt; t += PNT) {
      const int i = k + 1 + t / cnt, j = k + 1 + t % cnt;
      if (j <= i) Ab[(size_t)i * ld + (i - j)] -= Ab[(size_t)i * ld + (i - k)] * Ab[(size_t)j * ld + (j - k)];
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < n; c += PNT) {
    for (int i = 0; i < n; ++i) {  // L y = e_c
      double s = i == c ? 1.0 : 0.0;
      for (int j = max(0, i - bw); j < i; ++j) s -= Ab[(size_t)i * ld + (i - j)] * Kinv[(size_t)j * n + c];
      Kinv[(size_t)i * n + c] = s / Ab[(size_t)i * ld];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T x = y
      double s = Kinv[(size_t)i * n + c];
      for (int j = i + 1; j <= min(n - 1, i + bw); ++j) s -= Ab[(size_t)j * ld + (j - i)] * Kinv[(size_t)j * n + c];
      Kinv[(size_t)i * n + c] = s / Ab[(size_t)i * ld];
    }
  }
}

}  // namespace

struct mto_poisson {
  int device = 0, nelx = 0, nely = 0, L = 0, fl = 0, C = 1, n0 = 0;
  bool mixed = false;  // float32 V-cycle
  mto_poisson_opts o{};
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_a = nullptr, ev_b = nullptr;
  double* Kinv = nullptr;
  double* Ab = nullptr;
  int* err = nullptr;
  // Per right-hand-side workspace (grown on demand): r, p, q of the finest
  // grid and z[0], z[1], b of every grid, zero on the boundary.
  int cap = 0;
  double* ws = nullptr;
  size_t ws_per_rhs = 0;
  PDesc* d_desc = nullptr;
  PStats* d_stats = nullptr;
  PStats* h_stats = nullptr;  // pinned
  // Descriptors are staged from pageable memory: the copy call returns once
  // they have left this buffer, so that a later call may refill it at once.
  std::vector<PDesc> h_desc;
  std::vector<int> lvl_nodes;  // nodes of each grid
  long long launches = 0;
  mto_solve_stats last{};
  float ms_setup = 0.f;
};

namespace {

size_t level_nodes(int nx, int ny) { return (size_t)(nx + 1) * (ny + 1); }

// Workspace offsets (in doubles) of one right-hand side.
struct WsLayout {
  size_t r, p, q, z0[PMAXL], z1[PMAXL], b[PMAXL], total;
};
WsLayout ws_layout(const mto_poisson* c) {
  WsLayout w{};
  size_t off = 0;
  const size_t nf = c->lvl_nodes[c->L];
  w.r = off; off += nf;
  w.p = off; off += nf;
  w.q = off; off += nf;
  for (int l = 0; l <= c->L; ++l) {
    const size_t n = c->lvl_nodes[l];
    w.z0[l] = off; off += n;
    w.z1[l] = off; off += n;
    w.b[l] = off; off += n;
  }
  w.total = (off + 31) & ~(size_t)31;  // 256-byte aligned slices
  return w;
}

mto_status fail_cuda(cudaError_t e) {
  mto::g_last_cuda = e;
  cudaGetLastError();
  return MTO_ERR_CUDA;
}

#define PCK(call)                                \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return fail_cuda(e_); \
  } while (0)

mto_status grow_ws(mto_poisson* c, int n_rhs) {
  if (n_rhs <= c->cap) return MTO_OK;
  const WsLayout w = ws_layout(c);
  double* ws = nullptr;
  if (mto::device_alloc((void**)&ws, sizeof(double) * w.total * n_rhs) != cudaSuccess) {
    cudaGetLastError();
    return MTO_ERR_OOM;
  }
  // Boundary entries are never written by the kernel: zero them once (on
  // the legacy stream, which the solver's non-blocking stream does not order
  // against, so wait for it).
  if (cudaMemset(ws, 0, sizeof(double) * w.total * n_rhs) != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess) {
    mto::device_free(ws);
    return fail_cuda(cudaGetLastError());
  }
  PDesc* dd = nullptr;
  PStats* ds = nullptr;
  if (mto::device_alloc((void**)&dd, sizeof(PDesc) * n_rhs) != cudaSuccess ||
      mto::device_alloc((void**)&ds, sizeof(PStats) * n_rhs) != cudaSuccess) {
    cudaGetLastError();
    mto::device_free(ws);
    if (dd) mto::device_free(dd);
    return MTO_ERR_OOM;
  }
  PStats* hs = nullptr;
  if (cudaMallocHost(&hs, sizeof(PStats) * n_rhs) != cudaSuccess) {
    cudaGetLastError();
    mto::device_free(ws);
    mto::device_free(dd);
    mto::device_free(ds);
    return MTO_ERR_OOM;
  }
  cudaStreamSynchronize(c->stream);
  if (c->ws) mto::device_free(c->ws);
  if (c->d_desc) mto::device_free(c->d_desc);
  if (c->d_stats) mto::device_free(c->d_stats);
  if (c->h_stats) cudaFreeHost(c->h_stats);
  c->ws = ws;
  c->d_desc = dd;
  c->d_stats = ds;
  c->h_desc.resize(n_rhs);
  c->h_stats = hs;
  c->ws_per_rhs = w.total;
  c->cap = n_rhs;
  return MTO_OK;
}

// Descriptor of right-hand side k.
PDesc make_desc(const mto_poisson* c, int k, int mode, const double* in, double* out) {
  const WsLayout w = ws_layout(c);
  double* base = c->ws + c->ws_per_rhs * k;
  PDesc d;
  std::memset(&d, 0, sizeof(d));
  d.L = c->L;
  d.fl = c->fl;
  d.mode = mode;
  d.nu1 = c->o.nu1;
  d.nu2 = c->o.nu2;
  d.max_it = c->o.max_it;
  d.flexible = c->mixed ? 1 : 0;
  d.tol2 = c->o.tol * c->o.tol;
  d.wd = c->o.omega * 3.0 / 8.0;
  d.n0 = c->n0;
  d.Kinv = c->Kinv;
  d.f = in;
  d.x = out;
  d.r = base + w.r;
  d.p = base + w.p;
  d.q = base + w.q;
  d.stats = c->d_stats + k;
  for (int l = 0; l <= c->L; ++l) {
    const int sh = c->L - l;
    d.lv[l].nx = c->nelx >> sh;
    d.lv[l].ny = c->nely >> sh;
    d.lv[l].z[0] = base + w.z0[l];
    d.lv[l].z[1] = base + w.z1[l];
    d.lv[l].b = base + w.b[l];
  }
  return d;
}

// Enqueues one launch: a cluster of C CTAs per right-hand side.
mto_status launch(mto_poisson* c, int n, int mode, const double* in, double* out, size_t stride) {
  for (int k = 0; k < n; ++k) c->h_desc[k] = make_desc(c, k, mode, in + stride * k, out + stride * k);
  PCK(cudaMemcpyAsync(c->d_desc, c->h_desc.data(), sizeof(PDesc) * n, cudaMemcpyHostToDevice,
                      c->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->C * n);
  cfg.blockDim = dim3(PNT);
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = c->C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  c->launches += 1;
  if (c->mixed)
    PCK(cudaLaunchKernelEx(&cfg, poisson_cluster_kernel<float>, (const PDesc*)c->d_desc, c->C));
  else
    PCK(cudaLaunchKernelEx(&cfg, poisson_cluster_kernel<double>, (const PDesc*)c->d_desc, c->C));
  return MTO_OK;
}

mto_status enter(mto_poisson* c) {
  PCK(cudaSetDevice(c->device));
  PCK(cudaEventRecord(c->ev_in, c->user_stream));
  PCK(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  return MTO_OK;
}

mto_status leave(mto_poisson* c) {
  PCK(cudaEventRecord(c->ev_out, c->stream));
  PCK(cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
  return MTO_OK;
}

// Largest cluster size (power of two, <= want) that the device can schedule
// for the kernel of V-cycle type VT.
template <typename VT> int usable_cluster(int want) {
  cudaFuncSetAttribute(poisson_cluster_kernel<VT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
  for (int C = want; C > 1; C >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(PNT);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, poisson_cluster_kernel<VT>, &cfg) == cudaSuccess &&
        clusters > 0)
      return C;
    cudaGetLastError();
  }
  return 1;
}

}  // namespace

extern "C" {

void mto_poisson_default_opts(mto_poisson_opts* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->max_it = 500;
  o->omega = 0.6;
  o->nu1 = 2;
  o->nu2 = 2;
  o->n_coarsen = 3;
  o->cluster_ctas = 0;
  o->precision = MTO_PRECISION_FP64;
}

void mto_poisson_destroy(mto_poisson* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->ws) mto::device_free(c->ws);
  if (c->d_desc) mto::device_free(c->d_desc);
  if (c->d_stats) mto::device_free(c->d_stats);
  if (c->h_stats) cudaFreeHost(c->h_stats);
  if (c->Kinv) mto::device_free(c->Kinv);
  if (c->Ab) mto::device_free(c->Ab);
  if (c->err) mto::device_free(c->err);
  for (cudaEvent_t e : {c->ev_in, c->ev_out, c->ev_a, c->ev_b})
    if (e) cudaEventDestroy(e);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

static mto_status poisson_create_impl(mto_poisson* c, int device, void* stream) {
  PCK(cudaSetDevice(device));
  c->device = device;
  c->user_stream = static_cast<cudaStream_t>(stream);
  PCK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  PCK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  PCK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  PCK(cudaEventCreate(&c->ev_a));
  PCK(cudaEventCreate(&c->ev_b));
  // Cluster size: one CTA while the finest grid has at most LOCAL_MAX_NODES
  // interior nodes, else about one CTA per LOCAL_MAX_NODES of them (a power
  // of two, at most 16, at most what the device schedules): the float64 pipe
  // of one SM is the bound, so the work is spread as wide as the cluster
  // allows.
  const long long interior = (long long)(c->nelx - 1) * (c->nely - 1);
  int want = c->o.cluster_ctas;
  if (want == 0) {
    want = 1;
    while (want < PMAXC && (long long)want * LOCAL_MAX_NODES < interior) want <<= 1;
  }
  if (interior <= LOCAL_MAX_NODES) want = 1;
  c->C = want > 1 ? (c->mixed ? usable_cluster<float>(want) : usable_cluster<double>(want)) : 1;
  // Levels small enough for CTA 0 alone.
  c->fl = c->L;
  if (c->C > 1) {
    c->fl = 0;
    for (int l = 0; l < c->L; ++l) {
      const int sh = c->L - l;
      if ((long long)((c->nelx >> sh) - 1) * ((c->nely >> sh) - 1) <= LOCAL_MAX_NODES) c->fl = l;
    }
  }
  for (int l = 0; l <= c->L; ++l) {
    const int sh = c->L - l;
    c->lvl_nodes.push_back((int)level_nodes(c->nelx >> sh, c->nely >> sh));
  }
  // Coarsest grid: band Cholesky and explicit inverse on the device.
  const int nx0 = c->nelx >> c->L, ny0 = c->nely >> c->L;
  c->n0 = (nx0 - 1) * (ny0 - 1);
  const int ld = nx0 + 1;  // band width + 1
  if (mto::device_alloc((void**)&c->Kinv, sizeof(double) * (size_t)c->n0 * c->n0) != cudaSuccess ||
      mto::device_alloc((void**)&c->Ab, sizeof(double) * (size_t)c->n0 * ld) != cudaSuccess ||
      mto::device_alloc((void**)&c->err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return MTO_ERR_OOM;
  }
  PCK(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
  PCK(cudaEventRecord(c->ev_a, c->stream));
  poisson_coarsest_kernel<<<1, PNT, 0, c->stream>>>(nx0, ny0, c->Ab, c->Kinv, c->err);
  PCK(cudaGetLastError());
  c->launches += 1;
  PCK(cudaEventRecord(c->ev_b, c->stream));
  int err = 0;
  PCK(cudaMemcpyAsync(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PCK(cudaStreamSynchronize(c->stream));
  PCK(cudaEventElapsedTime(&c->ms_setup, c->ev_a, c->ev_b));
  if (err) return MTO_ERR_BREAKDOWN;
  return grow_ws(c, 1);
}

mto_status mto_poisson_create(mto_poisson** out, int nelx, int nely, const mto_poisson_opts* opts,
                              int device, void* cuda_stream) {
  mto::NvtxRange nvtx_range("mto_poisson_create");
  if (!out) return MTO_ERR_ARG;
  *out = nullptr;
  mto_poisson_opts o;
  mto_poisson_default_opts(&o);
  if (opts) o = *opts;
  const bool cl_ok = o.cluster_ctas == 0 || o.cluster_ctas == 1 || o.cluster_ctas == 2 ||
                     o.cluster_ctas == 4 || o.cluster_ctas == 8 || o.cluster_ctas == 16;
  if (nelx < 2 || nely < 2 || device < 0 || !(o.tol >= 0.0) || o.max_it < 0 || !(o.omega > 0.0) ||
      !(o.omega <= 1.0) || o.nu1 < 1 || o.nu2 < 1 || o.nu1 > 16 || o.nu2 > 16 || o.n_coarsen < 1 ||
      o.n_coarsen >= PMAXL || !cl_ok ||
      (o.precision != MTO_PRECISION_FP64 && o.precision != MTO_PRECISION_MIXED))
    return MTO_ERR_ARG;
  if (nelx % (1 << o.n_coarsen) || nely % (1 << o.n_coarsen)) return MTO_ERR_UNSUPPORTED_MESH;
  const int nx0 = nelx >> o.n_coarsen, ny0 = nely >> o.n_coarsen;
  if (nx0 < 2 || ny0 < 2 || (long long)(nx0 - 1) * (ny0 - 1) > PMAX_COARSE ||
      (long long)(nelx + 1) * (nely + 1) > (1LL << 28))
    return MTO_ERR_UNSUPPORTED_MESH;
  mto_poisson* c = new (std::nothrow) mto_poisson();
  if (!c) return MTO_ERR_OOM;
  c->nelx = nelx;
  c->nely = nely;
  c->o = o;
  c->L = o.n_coarsen;
  c->mixed = o.precision == MTO_PRECISION_MIXED;
  const mto_status s = poisson_create_impl(c, device, cuda_stream);
  if (s != MTO_OK) {
    cudaGetLastError();
    mto_poisson_destroy(c);
    return s;
  }
  *out = c;
  return MTO_OK;
}

mto_status mto_poisson_solve(mto_poisson* c, int n_rhs, const double* f_dev, double* u_dev,
                             mto_solve_stats* stats) {
  mto::NvtxRange nvtx_range("mto_poisson_solve");
  if (!c || !f_dev || !u_dev || n_rhs < 1 || n_rhs > PMAX_RHS) return MTO_ERR_ARG;
  mto_status s = enter(c);
  if (s != MTO_OK) return s;
  if ((s = grow_ws(c, n_rhs)) != MTO_OK) return s;
  PCK(cudaEventRecord(c->ev_a, c->stream));
  if ((s = launch(c, n_rhs, PMODE_SOLVE, f_dev, u_dev, c->lvl_nodes[c->L])) != MTO_OK) return s;
  PCK(cudaEventRecord(c->ev_b, c->stream));
  PCK(cudaMemcpyAsync(c->h_stats, c->d_stats, sizeof(PStats) * n_rhs, cudaMemcpyDeviceToHost,
                      c->stream));
  PCK(cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  PCK(cudaEventElapsedTime(&ms, c->ev_a, c->ev_b));
  mto_status worst = MTO_OK;
  int total = 0;
  for (int k = 0; k < n_rhs; ++k) {
    const PStats& p = c->h_stats[k];
    total += p.iters;
    const mto_status sk = p.status == PST_CONVERGED ? MTO_OK
                          : p.status == PST_MAXIT   ? MTO_ERR_NOT_CONVERGED
                                                    : MTO_ERR_BREAKDOWN;
    if (sk != MTO_OK && worst == MTO_OK) worst = sk;
  }
  const PStats& p = c->h_stats[n_rhs - 1];
  const double fn = std::sqrt(p.ff);
  c->last.iters = total;
  c->last.converged = worst == MTO_OK;
  c->last.rel_res_rec = fn > 0 ? std::sqrt(p.rr) / fn : 0.0;
  c->last.rel_res_true = fn > 0 ? std::sqrt(p.rr_true) / fn : 0.0;
  c->last.ms_solve = ms;
  c->last.ms_setup = c->ms_setup;
  if (stats) *stats = c->last;
  if ((s = leave(c)) != MTO_OK) return s;
  return worst;
}

mto_status mto_poisson_apply_operator(mto_poisson* c, const double* v_dev, double* y_dev) {
  if (!c || !v_dev || !y_dev) return MTO_ERR_ARG;
  mto_status s = enter(c);
  if (s != MTO_OK) return s;
  if ((s = launch(c, 1, PMODE_APPLY, v_dev, y_dev, 0)) != MTO_OK) return s;
  return leave(c);
}

mto_status mto_poisson_apply_preconditioner(mto_poisson* c, const double* r_dev, double* z_dev) {
  if (!c || !r_dev || !z_dev) return MTO_ERR_ARG;
  mto_status s = enter(c);
  if (s != MTO_OK) return s;
  if ((s = launch(c, 1, PMODE_PRECOND, r_dev, z_dev, 0)) != MTO_OK) return s;
  return leave(c);
}

mto_status mto_poisson_get_info(mto_poisson* c, int* n_levels, int* coarsest_free, int* cluster_ctas,
                                long long* launches) {
  if (!c) return MTO_ERR_ARG;
  if (n_levels) *n_levels = c->L + 1;
  if (coarsest_free) *coarsest_free = c->n0;
  if (cluster_ctas) *cluster_ctas = c->C;
  if (launches) *launches = c->launches;
  return MTO_OK;
}

}  // extern "C"
