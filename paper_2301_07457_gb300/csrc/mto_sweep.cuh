// Matrix-free stencil sweeps of the V-cycle and the outer CG operator.
//
// One warp owns a strip of node columns and a chunk of rows.  Lane L holds
// node column i and marches upwards one element row per step: it takes the
// node values of the new top row (the right neighbour's by shuffle), forms
// the element (i, je) to its right once, and completes node row je.  Lanes
// 1..30 own complete columns; lanes 0 and 31 are halo columns shared with the
// neighbouring strips, so every lane runs the same instructions (no
// single-lane paths, which would cost a full warp slot on the FP64 pipe).
// Every element is evaluated 32/30 times overall, every node value is read
// once plus one halo row per chunk, and there is no shared memory and no
// atomics.  Loads run PF steps ahead of the arithmetic (a register ring), so
// each warp keeps PF rows of memory traffic in flight; addresses advance by
// one row pitch per step.
//
// The element operator works on edges (see mto_common.cuh for the strain
// basis).  Per element: the top-edge differences b, the left-edge differences
// dl (the right edge comes from the next lane, the bottom edge is the previous
// step's top edge), then c1 = a + b, c3 = b - a, c2 = dl + dr (u_x) and the
// same for u_y; after the 5x5 core, the forces go back through the edges:
// a horizontal edge collects ga = t_c1 - t_c3 from the element above it and
// gb = t_c1 + t_c3 from the element below, a vertical edge collects t_s (u_x)
// or t_d2 (u_y) from its two elements, and a node sums its four edges with
// signs.  That is 11 + 14 add/sub per node plus the core, about a third fewer
// operations than forming the four corner forces of every element.
//
// Modes (all masked by the clamped edges; ghost nodes are zero by layout):
//   APPLY    out = K v
//   RESID    out = b - K v,                        dot |out|^2
//   KP       p = z + beta p_old, q = K p,           dot p.q      (Alg. 2)
//   SMOOTH   out = v + w D^-1 (b - K v)                           (Sec. 2.3)
//   SMOOTH0  as SMOOTH with v = w D^-1 b formed on the fly (first sweep
//            from zero followed by the second, Alg. 1 pre-smoothing)
//   PSMOOTH  v' = v + P zc (Alg. 1 correction), out = v' + w D^-1 (b - K v')
//   RESTRICT bc = P^T (b - K v) on the next coarser grid          (Alg. 1)
// SMOOTH/PSMOOTH optionally accumulate z.r (and z.q for the flexible beta).
#pragma once

#include "mto_common.cuh"

namespace mto {

constexpr int SWEEP_NT = 256;
// Output columns per warp: 30 (lanes 1..30) for the stencil modes, 28 fine
// columns = 14 coarse columns for the restriction.
constexpr int SWEEP_STRIDE = 30;
constexpr int SWEEP_RSTRIDE = 28;

// SRC_CFINE: the first coarse level of the mixed path, whose Galerkin element
// matrices are rebuilt on the fly from the four bf16 fine moduli they cover
// (8 bytes per coarse element instead of 13 stored coefficients).
// SRC_CMOM: the deeper float32 coarse levels, which store the six scaled
// moments of each element (24 bytes) and form the 13 coefficients in
// registers.
enum Src { SRC_FINE64 = 0, SRC_FINEBF = 1, SRC_COARSE = 2, SRC_CFINE = 3, SRC_CMOM = 4 };
enum Mode {
  MODE_APPLY = 0,
  MODE_RESID,
  MODE_KP,
  MODE_SMOOTH,
  MODE_PSMOOTH,
  MODE_RESTRICT,
  MODE_SMOOTH0,
  MODE_POST2,  // float32 coarse levels: prolongation + two sweeps, fused (mto_fused.cuh)
  MODE_PRE2    // float32 coarse levels: two sweeps from zero + residual + restriction, fused
};

template <typename T> struct SweepParams {
  using T2 = typename V2<T>::t;
  Grid g;   // this level
  Grid gc;  // next coarser level (PSMOOTH source, RESTRICT target)
  int nstrips, nchunks, H;
  int gate;          // 1: skip the launch once the PCG has stopped (sc->done)
  int replace_gate;  // RESID as residual replacement: run only when iter % rr_every == 0
  int zero_gate;     // RESID of the initial guess: out = b when sc->x_nonzero == 0 (K 0 = 0)
  const T2* v;       // marched vector (z, x or p_old)
  const T2* zc;      // PSMOOTH: coarse correction
  const void* zkp;   // KP: z (double2 or float2)
  T2* p_out;         // KP: new search direction
  T2* xvec;          // KP: the iterate x, advanced by the pending step alpha p_old (x_lag)
  const T2* xdir;    // RESID with xlag: the direction p of the pending step
  int xlag;          // RESID: apply the pending step to v on the fly (v = x + alpha p) when x_lag
  int tag;           // KP: index of p_out among the two search-direction buffers
  const T2* b;       // right-hand side (SMOOTH, SMOOTH0, PSMOOTH, RESTRICT, RESID)
  T2* out;           // output vector (APPLY, RESID, KP: q, SMOOTH*, PSMOOTH)
  float2* out32;     // RESID: optional float32 copy of out (the mixed V-cycle's input)
  T2* bc;            // RESTRICT: coarse right-hand side
  const void* E;     // finest level: 4 scaled float64 moduli per element (FINE64) or bf16 E
  const T* coef;     // coarse element matrices, NCOEF arrays of g.size() (SRC_CMOM: NMOM moments)
  long long cstride;
  T cnu, cg;         // SRC_CMOM: nu and g = (1 - nu) / 2
  FineConst<T> kf;      // bf16 finest level / SRC_CFINE: scale factors of the element core
  Grid gfine;           // SRC_CFINE: the finer grid whose bf16 moduli E points to
  int redisc;           // SRC_CFINE: rediscretised (mean modulus) instead of Galerkin
  const double* invd1;  // float64 finest level: w / D per node
  const T2* invd2;      // coarse levels: w / D per DOF
  T wdiag;              // float32 finest level: w / (KE_00 at E = 1); D = sum of 4 moduli
  const double2* rdot;  // dot partner for z.r
  const double2* qdot;  // dot partner for z.q (flexible beta), may be null
  double2* r64;            // bf16 SMOOTH0 with the CG update: r of this step (written)
  const double2* r64_prev;  // ... r of the last step, read while the update is pending
  const double2* q64;       // ... and q = K p of the last step
  double* partials;
  unsigned* ticket;
  DevScalars* sc;
  int finish;
  double* out_value;
};

template <typename T2> __device__ __forceinline__ T2 shfl_down2(T2 v) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
  return v;
}
template <typename T2> __device__ __forceinline__ T2 shfl_up2(T2 v) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
  return v;
}
template <typename T2> __device__ __forceinline__ T2 add2(T2 a, T2 b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename T2> __device__ __forceinline__ T2 sub2(T2 a, T2 b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
// float2 pairs use Blackwell's packed FP32 instructions (two correctly
// rounded operations per instruction): the float32 sweeps are bound by
// instruction issue, and most of their arithmetic treats u_x and u_y alike.
__device__ __forceinline__ unsigned long long pk2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
template <> __device__ __forceinline__ float2 add2<float2>(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
template <> __device__ __forceinline__ float2 sub2<float2>(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
// a * b + c per component (float2: one packed FMA).
template <typename T2> __device__ __forceinline__ T2 fma2(T2 a, T2 b, T2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.y = fma(a.y, b.y, c.y);
  return c;
}
template <> __device__ __forceinline__ float2 fma2<float2>(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(r);
}
template <typename T2> __device__ __forceinline__ T2 mul2(T2 a, T2 b) {
  a.x *= b.x;
  a.y *= b.y;
  return a;
}
template <> __device__ __forceinline__ float2 mul2<float2>(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}

// Raw loads of the marched vector at one node (finished later, so that the
// loads can be in flight while earlier steps compute).
template <typename T, int MODE, typename ZT> struct VRaw {
  using T2 = typename V2<T>::t;
  T2 v;                  // z, p_old, x, or b (SMOOTH0)
  ZT z;                  // KP: z
  T2 c00, c10, c01, c11; // PSMOOTH: coarse corners
  double d1;             // SMOOTH0 on the float64 finest level: w / D
  T2 d2;                 // SMOOTH0 on a coarse level: w / D
};

template <typename T, int SRC> struct ERaw;
template <typename T> struct ERaw<T, SRC_FINE64> {
  double2 k01, k23;  // E kA, E kB, E kC, E kG
};
template <typename T> struct ERaw<T, SRC_FINEBF> {
  __nv_bfloat16 E;
};
template <typename T> struct ERaw<T, SRC_COARSE> {
  T A[NCOEF];
};
template <typename T> struct ERaw<T, SRC_CFINE> {
  __nv_bfloat162 lo, hi;  // fine moduli of rows 2J and 2J+1, columns 2I and 2I+1
};
template <typename T> struct ERaw<T, SRC_CMOM> {
  T m[NMOM];
};

// Loads that belong to the node row being completed.
template <typename T> struct NRaw {
  using T2 = typename V2<T>::t;
  T2 b;
  T2 d2;
  double d1;
  double2 rd, qd;
};

template <typename T, int SRC, int MODE, bool DOT, typename ZT> struct Sweep {
  using T2 = typename V2<T>::t;
  using VR = VRaw<T, MODE, ZT>;
  using ER = ERaw<T, SRC>;
  static constexpr bool NEEDS_B = MODE == MODE_RESID || MODE == MODE_SMOOTH ||
                                  MODE == MODE_SMOOTH0 || MODE == MODE_PSMOOTH ||
                                  MODE == MODE_RESTRICT;
  static constexpr bool SMOOTHING = MODE == MODE_SMOOTH || MODE == MODE_SMOOTH0 ||
                                    MODE == MODE_PSMOOTH;

  __device__ __forceinline__ static void load_v(const SweepParams<T>& a, long long k, int ii, int jj,
                                                VR& r) {
    if constexpr (MODE == MODE_KP) {
      r.z = static_cast<const ZT*>(a.zkp)[k];
      r.v = a.v[k];
    } else if constexpr (MODE == MODE_PSMOOTH) {
      r.v = a.v[k];
      // Clamp to a readable coarse node; invalid fine nodes are masked later.
      const int I0 = max(ii, 0) >> 1, J0 = max(jj, 0) >> 1;
      const Grid gc = a.gc;
      r.c00 = a.zc[gc.at(I0, J0)];
      r.c10 = a.zc[gc.at(I0 + 1, J0)];
      r.c01 = a.zc[gc.at(I0, J0 + 1)];
      r.c11 = a.zc[gc.at(I0 + 1, J0 + 1)];
    } else if constexpr (MODE == MODE_SMOOTH0) {
      r.v = a.b[k];
      if constexpr (SRC == SRC_FINE64) r.d1 = a.invd1[k];
      else r.d2 = a.invd2[k];
    } else {
      r.v = a.v[k];
    }
  }

  __device__ __forceinline__ static T2 finish_v(const SweepParams<T>& a, const VR& r, int ii, int jj,
                                                T beta) {
    if constexpr (MODE == MODE_KP) {
      if constexpr (sizeof(T) == 8) {
        return mk2<T>(to_f64(r.z.x) + beta * r.v.x, to_f64(r.z.y) + beta * r.v.y);
      } else {
        return mk2<T>(T(r.z.x) + beta * r.v.x, T(r.z.y) + beta * r.v.y);
      }
    } else if constexpr (MODE == MODE_PSMOOTH) {
      if (!a.g.valid(ii, jj)) return mk2<T>(T(0), T(0));
      const T wx0 = (ii & 1) ? T(0.5) : T(1), wx1 = (ii & 1) ? T(0.5) : T(0);
      const T wy0 = (jj & 1) ? T(0.5) : T(1), wy1 = (jj & 1) ? T(0.5) : T(0);
      const T ix = wy0 * (wx0 * r.c00.x + wx1 * r.c10.x) + wy1 * (wx0 * r.c01.x + wx1 * r.c11.x);
      const T iy = wy0 * (wx0 * r.c00.y + wx1 * r.c10.y) + wy1 * (wx0 * r.c01.y + wx1 * r.c11.y);
      return mk2<T>(r.v.x + ix, r.v.y + iy);
    } else if constexpr (MODE == MODE_SMOOTH0) {
      // w D^-1 is zero on clamped and ghost nodes, so no mask is needed.
      if constexpr (SRC == SRC_FINE64) return mk2<T>(T(r.d1) * r.v.x, T(r.d1) * r.v.y);
      else return mk2<T>(r.d2.x * r.v.x, r.d2.y * r.v.y);
    } else {
      return r.v;
    }
  }

  __device__ __forceinline__ static void load_e(const SweepParams<T>& a, long long e, int ii, int jj,
                                                ER& r) {
    if constexpr (SRC == SRC_CFINE) {
      // Ghost and padding elements have no children: zero operator.
      if ((unsigned)ii < (unsigned)a.g.nx && (unsigned)jj < (unsigned)a.g.ny) {
        const __nv_bfloat162* Ef = static_cast<const __nv_bfloat162*>(a.E);
        const long long kf = a.gfine.at(2 * ii, 2 * jj);  // even: bf16 pairs are aligned
        r.lo = Ef[kf >> 1];
        r.hi = Ef[(kf + a.gfine.pitch) >> 1];
      } else {
        r.lo = r.hi = __floats2bfloat162_rn(0.f, 0.f);
      }
    } else if constexpr (SRC == SRC_FINE64) {
      const double2* p = static_cast<const double2*>(a.E) + 2 * e;
      r.k01 = __ldg(p);
      r.k23 = __ldg(p + 1);
    } else if constexpr (SRC == SRC_FINEBF) {
      r.E = static_cast<const __nv_bfloat16*>(a.E)[e];
    } else if constexpr (SRC == SRC_CMOM) {
#pragma unroll
      for (int c = 0; c < NMOM; ++c) r.m[c] = a.coef[c * a.cstride + e];
    } else {
#pragma unroll
      for (int c = 0; c < NCOEF; ++c) r.A[c] = a.coef[c * a.cstride + e];
    }
  }

  __device__ __forceinline__ static void load_n(const SweepParams<T>& a, long long k, NRaw<T>& r) {
    if constexpr (NEEDS_B) r.b = a.b[k];
    if constexpr (SMOOTHING) {
      if constexpr (SRC == SRC_FINE64) r.d1 = a.invd1[k];
      else if constexpr (SRC == SRC_COARSE || SRC == SRC_CFINE || SRC == SRC_CMOM) r.d2 = a.invd2[k];
      if constexpr (DOT) {
        r.rd = a.rdot[k];
        if (a.qdot != nullptr) r.qd = a.qdot[k];
      }
    }
  }

  // Strain-space forces t = A w of one element.
  __device__ __forceinline__ static Strain<T> core(const SweepParams<T>& a, const ER& er,
                                                   const Strain<T>& w, T& Ecur) {
    Strain<T> t;
    if constexpr (SRC == SRC_FINE64) {
      const T eA = er.k01.x, eB = er.k01.y, eC = er.k23.x, eG = er.k23.y;
      t.c1 = eA * w.c1 + eB * w.d2;
      t.d2 = eA * w.d2 + eB * w.c1;
      t.c3 = eC * w.c3;
      t.d3 = eC * w.d3;
      t.s = eG * w.s;
    } else if constexpr (SRC == SRC_FINEBF) {
      Ecur = __bfloat162float(er.E);
      t = fine_core<T>(w, Ecur, a.kf);
    } else if constexpr (SRC == SRC_CFINE) {
      // Moments of the four child moduli (children at xi, eta = +-1/2 of the
      // parent): M00 = S/4, M10 = X/8, M01 = Y/8, M20 = M02 = M00/3,
      // M11 = Z/16, then the 13 coefficients of mto_common.cuh.
      const float2 l = __bfloat1622float2(er.lo), h = __bfloat1622float2(er.hi);
      const T e00 = l.x, e10 = l.y, e01 = h.x, e11 = h.y;
      const T M00 = T(0.25) * ((e00 + e10) + (e01 + e11));
      T M10 = T(0.125) * ((e10 + e11) - (e00 + e01));
      T M01 = T(0.125) * ((e01 + e11) - (e00 + e10));
      T M11 = T(0.0625) * ((e00 + e11) - (e10 + e01));
      if (a.redisc) M10 = M01 = M11 = T(0);
      const FineConst<T> k = a.kf;  // kappa, kappa nu, kappa (1+g)/3, kappa g
      T A[NCOEF];
      A[0] = k.kA * M00;
      A[1] = k.kA * M01;
      A[2] = k.kC * M00;
      A[3] = k.kA * M00;
      A[4] = k.kA * M10;
      A[5] = k.kC * M00;
      A[6] = k.kB * M00;
      A[7] = k.kB * M10;
      A[8] = k.kB * M01;
      A[9] = (k.kB + k.kG) * M11;
      A[10] = k.kG * M00;
      A[11] = k.kG * M10;
      A[12] = k.kG * M01;
      t = coarse_core<T>(w, A);
    } else if constexpr (SRC == SRC_CMOM) {
      T A[NCOEF];
      coefs_from_kmom<T>(er.m, a.cnu, a.cg, A);
      t = coarse_core<T>(w, A);
    } else {
      t = coarse_core<T>(w, er.A);
    }
    return t;
  }
};

template <typename T, int SRC, int MODE, bool DOT, typename ZT, int PF>
__global__ void __launch_bounds__(SWEEP_NT) sweep_kernel(const SweepParams<T> a) {
  using T2 = typename V2<T>::t;
  using S = Sweep<T, SRC, MODE, DOT, ZT>;
  using VR = typename S::VR;
  using ER = typename S::ER;
  // The bf16 finest level stores no w/D; its fused first sweep exists only
  // in the two-column kernel (mto_sweep2.cuh).
  static_assert(!(SRC == SRC_FINEBF && MODE == MODE_SMOOTH0), "use sweep2_kernel");
  constexpr bool REDUCE = DOT || MODE == MODE_RESID || MODE == MODE_KP;
  pdl_wait();
  if (a.sc != nullptr && a.gate) {
    if (a.sc->done != RUNNING) return;  // uniform over the grid
    if (a.replace_gate && (a.sc->rr_every <= 0 || (a.sc->iter % a.sc->rr_every) != 0)) return;
  }
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (SWEEP_NT / 32) + (threadIdx.x >> 5);
  const int strip = wg % a.nstrips;
  const int chunk = wg / a.nstrips;
  double dot0 = 0.0, dot1 = 0.0;
  T beta = T(0);
  if constexpr (MODE == MODE_KP) beta = T(a.sc->beta);
  bool vzero = false;
  if constexpr (MODE == MODE_RESID) vzero = a.zero_gate && a.sc->x_nonzero == 0;

  if (vzero) {
    // Residual of a zero iterate: r = b on the free DOFs, no operator needed.
    if (chunk < a.nchunks) {
      const Grid g = a.g;
      const int i = strip * SWEEP_STRIDE - 1 + lane;
      const bool own_col = lane >= 1 && lane <= 30 && i >= 0 && i <= g.nx;
      const int r0 = chunk * a.H, r1 = min(r0 + a.H - 1, g.ny);
      for (int j = r0; j <= r1 && own_col; ++j) {
        const long long k = g.at(i, j);
        T2 r = mk2<T>(T(0), T(0));
        if (!g.is_fixed(i, j)) r = a.b[k];
        a.out[k] = r;
        if (a.out32 != nullptr) a.out32[k] = make_float2(float(r.x), float(r.y));
        dot0 = fma(double(r.x), double(r.x), fma(double(r.y), double(r.y), dot0));
      }
    }
  } else if (chunk < a.nchunks) {
    constexpr int STRIDE = MODE == MODE_RESTRICT ? SWEEP_RSTRIDE : SWEEP_STRIDE;
    constexpr int SHIFT = MODE == MODE_RESTRICT ? 2 : 1;
    const Grid g = a.g;
    const int i = strip * STRIDE - SHIFT + lane;
    int je0, je1, Jb = 0, Je = 0;
    if constexpr (MODE == MODE_RESTRICT) {
      Jb = chunk * (a.H >> 1);
      Je = min(Jb + (a.H >> 1) - 1, a.gc.ny);
      je0 = max(2 * Jb - 2, -1);
      je1 = 2 * Je + 1;
    } else {
      const int r0 = chunk * a.H;
      je0 = r0 - 1;
      je1 = min(r0 + a.H - 1, g.ny);
    }
    // Column facts of this lane, fixed for the whole march.
    const bool own_col = lane >= 1 && lane <= 30 && i >= 0 && i <= g.nx;
    const bool col_fixed = ((g.fixed & 2u) && i == 0) || ((g.fixed & 4u) && i == g.nx);
    const long long pitch = g.pitch;

    struct Pack {
      VR vt;
      ER e;
      NRaw<T> n;
    };
    // Offsets of node (i, je + 1) and element / node (i, je) for step je.
    auto load_pack = [&](Pack& pk, int je, long long ke) {
      S::load_v(a, ke + pitch, i, je + 1, pk.vt);
      S::load_e(a, ke, i, je, pk.e);
      S::load_n(a, ke, pk.n);
    };

    const long long k0 = g.at(i, je0);
    // Marched values of the first row.
    T2 vb;
    {
      VR r0;
      S::load_v(a, k0, i, je0, r0);
      vb = S::finish_v(a, r0, i, je0, beta);
    }
    T2 vbr = shfl_down2(vb);
    T2 acarry = sub2(vbr, vb);  // bottom-edge differences of the current element row
    T2 gbprev = mk2<T>(T(0), T(0)), gvprev = gbprev;
    T Eprev = T(0);
    T2 racc = mk2<T>(T(0), T(0));  // RESTRICT: partial coarse row

    Pack ring[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u)
      if (je0 + u <= je1) load_pack(ring[u], je0 + u, k0 + u * pitch);

    long long k = k0;  // offset of node / element (i, je)
    for (int jb = je0; jb <= je1; jb += PF) {
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int je = jb + u;
        if (je > je1) break;
        const Pack cur = ring[u];
        if (je + PF <= je1) load_pack(ring[u], je + PF, k + PF * pitch);

        // ---- element (i, je) from rows je (vb, vbr) and je + 1 (vt, vtr) ----
        const T2 vt = S::finish_v(a, cur.vt, i, je + 1, beta);
        const T2 vtr = shfl_down2(vt);  // lane 31: its own value, never used for output
        const T2 bt = sub2(vtr, vt);    // top-edge differences
        const T2 dl = sub2(vt, vb);     // left-edge differences
        const T2 dr = shfl_down2(dl);   // right edge = next lane's left edge
        Strain<T> w;
        w.c1 = acarry.x + bt.x;
        w.c3 = bt.x - acarry.x;
        const T c2 = dl.x + dr.x;
        const T d1 = acarry.y + bt.y;
        w.d3 = bt.y - acarry.y;
        w.d2 = dl.y + dr.y;
        w.s = c2 + d1;
        T Ecur = T(0);
        const Strain<T> t = S::core(a, cur.e, w, Ecur);
        // ---- edge forces and node row je ----
        const T2 ga = mk2<T>(t.c1 - t.c3, t.s - t.d3);  // bottom edge of this element
        const T2 gb = mk2<T>(t.c1 + t.c3, t.s + t.d3);  // top edge of this element
        const T2 gh = add2(ga, gbprev);                 // horizontal edge (i, je) -> (i+1, je)
        const T2 gsv = mk2<T>(t.s, t.d2);
        const T2 gv = add2(gsv, shfl_up2(gsv));         // vertical edge (i, je) -> (i, je+1)
        const T2 ghl = shfl_up2(gh);
        const T2 kv = mk2<T>((ghl.x - gh.x) + (gvprev.x - gv.x), (ghl.y - gh.y) + (gvprev.y - gv.y));
        T eol = T(0), eo = T(0);
        if constexpr (SRC == SRC_FINEBF && S::SMOOTHING) {
          eo = Eprev + Ecur;
          eol = __shfl_up_sync(0xffffffffu, eo, 1);
          Eprev = Ecur;
        }
        const bool inb = je > je0 && own_col && je >= 0 && je <= g.ny;
        const bool act = inb && !col_fixed && !(((g.fixed & 1u) && je == 0) || ((g.fixed & 8u) && je == g.ny));
        if constexpr (MODE == MODE_APPLY) {
          if (inb) a.out[k] = act ? kv : mk2<T>(T(0), T(0));
        } else if constexpr (MODE == MODE_RESID) {
          T2 r = mk2<T>(T(0), T(0));
          if (act) r = sub2(cur.n.b, kv);
          if (inb) a.out[k] = r;
          if (inb && a.out32 != nullptr) a.out32[k] = make_float2(float(r.x), float(r.y));
          dot0 = fma(double(r.x), double(r.x), fma(double(r.y), double(r.y), dot0));
        } else if constexpr (MODE == MODE_KP) {
          const T2 q = act ? kv : mk2<T>(T(0), T(0));
          if (inb) {
            a.p_out[k] = vb;
            a.out[k] = q;
          }
          if (inb) dot0 = fma(double(vb.x), double(q.x), fma(double(vb.y), double(q.y), dot0));
        } else if constexpr (S::SMOOTHING) {
          T2 zn = mk2<T>(T(0), T(0));
          if (act) {
            const T2 res = sub2(cur.n.b, kv);
            T dx, dy;
            if constexpr (SRC == SRC_FINE64) {
              dx = dy = T(cur.n.d1);
            } else if constexpr (SRC == SRC_FINEBF) {
              dx = dy = __fdividef(a.wdiag, eo + eol);
            } else {  // coarse levels: stored w / D
              dx = cur.n.d2.x;
              dy = cur.n.d2.y;
            }
            zn = mk2<T>(vb.x + dx * res.x, vb.y + dy * res.y);
          }
          if (inb) a.out[k] = zn;
          if constexpr (DOT) {
            if (act) {
              const double zx = to_f64(zn.x), zy = to_f64(zn.y);
              dot0 = fma(zx, cur.n.rd.x, fma(zy, cur.n.rd.y, dot0));
              if (a.qdot != nullptr) dot1 = fma(zx, cur.n.qd.x, fma(zy, cur.n.qd.y, dot1));
            }
          }
        } else if constexpr (MODE == MODE_RESTRICT) {
          T2 r = mk2<T>(T(0), T(0));
          if (act) r = sub2(cur.n.b, kv);
          // Horizontal full weighting (1/2, 1, 1/2) by shuffles, then vertical
          // accumulation along the march.  Producers are the even lanes 2..28,
          // whose neighbours (lanes 1..29) hold complete residuals.
          const T2 ru = shfl_up2(r), rd = shfl_down2(r);
          const T2 h = mk2<T>(r.x + T(0.5) * (ru.x + rd.x), r.y + T(0.5) * (ru.y + rd.y));
          if (je > je0) {
            if (je & 1) {
              const int Jlo = (je - 1) / 2;
              const T2 val = mk2<T>(racc.x + T(0.5) * h.x, racc.y + T(0.5) * h.y);
              const bool producer = (lane & 1) == 0 && lane >= 2 && lane <= 28;
              const int I = i >> 1;
              if (producer && Jlo >= Jb && Jlo <= Je && I >= 0 && I <= a.gc.nx) {
                a.bc[a.gc.at(I, Jlo)] = a.gc.is_fixed(I, Jlo) ? mk2<T>(T(0), T(0)) : val;
              }
              racc = mk2<T>(T(0.5) * h.x, T(0.5) * h.y);
            } else {
              racc = add2(racc, h);
            }
          }
        }
        acarry = bt;
        gbprev = gb;
        gvprev = gv;
        vb = vt;
        k += pitch;
      }
    }
  }
  if constexpr (REDUCE) {
    block_reduce_finish<SWEEP_NT>(dot0, dot1, a.partials, a.ticket, a.sc, a.finish, a.out_value);
  }
}

}  // namespace mto
