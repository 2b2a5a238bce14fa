// Marching sweeps with two node columns per lane.
//
// Same operator, modes and edge-force bookkeeping as mto_sweep.cuh; only the
// mapping of lanes to columns differs.  Lane L holds the node columns
// i0 = base + 2L (even) and i1 = i0 + 1 and forms two elements per step:
// (i0, je), whose four corners it holds, and (i1, je), whose right corners
// come from the next lane by shuffle.  Lane 0's column i0 and lane 31's
// column i1 are halo columns, so a warp completes 62 columns (60 fine columns
// = 30 coarse columns for the restriction) instead of 30, a node pair moves in
// one 16-byte access, and the shuffles, address updates, masks and loop
// control of a step are shared by two nodes.  That matters for the float32
// sweeps, whose cost is instruction issue rather than DRAM bandwidth.
//
// Row pipelines (one step = one element row je, completing node row je):
//   * node values of row je + 1 (loaded PF steps ahead);
//   * element data of row je, except the bf16 finest moduli, which run one
//     row ahead (row je + 1) so that SMOOTH0 can form D at the top row;
//   * node-row data of row je (right-hand side, w/D, dot partners).
// SMOOTH0 carries the right-hand side and w/D of the top row into the next
// step instead of loading them twice.
#pragma once

#include "mto_sweep.cuh"

namespace mto {

constexpr int SWEEP2_STRIDE = 62;
constexpr int SWEEP2_RSTRIDE = 60;

// ---- node-pair access (k even: 16-byte aligned for float2, 32 for double2) ----
__device__ __forceinline__ void ld_pair(const float2* p, long long k, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p + k);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, long long k, double2& a, double2& b) {
  a = p[k];
  b = p[k + 1];
}
__device__ __forceinline__ void st_pair(float2* p, long long k, float2 a, float2 b, bool w0,
                                        bool w1) {
  if (w0 && w1) {
    *reinterpret_cast<float4*>(p + k) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    if (w0) p[k] = a;
    if (w1) p[k + 1] = b;
  }
}
__device__ __forceinline__ void st_pair(double2* p, long long k, double2 a, double2 b, bool w0,
                                        bool w1) {
  if (w0) p[k] = a;
  if (w1) p[k + 1] = b;
}

// L2 prefetch hint for the 32 bytes of a pair (no registers, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Element data of the pair (i0, j), (i1, j).
template <typename T, int SRC> struct ERaw2;
template <typename T> struct ERaw2<T, SRC_FINE64> {
  double2 k[4];  // element i0: k[0], k[1]; element i1: k[2], k[3]
};
template <typename T> struct ERaw2<T, SRC_FINEBF> {
  __nv_bfloat162 E;
  __nv_bfloat162 El;  // SMOOTH0: elements i0 - 2, i0 - 1
};
template <typename T> struct ERaw2<T, SRC_COARSE> {
  typename V2<T>::t A[NCOEF];
};
template <typename T> struct ERaw2<T, SRC_CFINE> {
  __nv_bfloat162 lo[2], hi[2];  // fine moduli of rows 2J, 2J+1; [w] = coarse element i0 + w
};
template <typename T> struct ERaw2<T, SRC_CMOM> {
  typename V2<T>::t m[NMOM];
};

template <typename T>
__device__ __forceinline__ ERaw<T, SRC_FINE64> pick(const ERaw2<T, SRC_FINE64>& r, int w) {
  ERaw<T, SRC_FINE64> e;
  e.k01 = w ? r.k[2] : r.k[0];
  e.k23 = w ? r.k[3] : r.k[1];
  return e;
}
template <typename T>
__device__ __forceinline__ ERaw<T, SRC_COARSE> pick(const ERaw2<T, SRC_COARSE>& r, int w) {
  ERaw<T, SRC_COARSE> e;
#pragma unroll
  for (int c = 0; c < NCOEF; ++c) e.A[c] = w ? r.A[c].y : r.A[c].x;
  return e;
}
template <typename T>
__device__ __forceinline__ ERaw<T, SRC_CMOM> pick(const ERaw2<T, SRC_CMOM>& r, int w) {
  ERaw<T, SRC_CMOM> e;
#pragma unroll
  for (int c = 0; c < NMOM; ++c) e.m[c] = w ? r.m[c].y : r.m[c].x;
  return e;
}
template <typename T>
__device__ __forceinline__ ERaw<T, SRC_CFINE> pick(const ERaw2<T, SRC_CFINE>& r, int w) {
  ERaw<T, SRC_CFINE> e;
  e.lo = r.lo[w];
  e.hi = r.hi[w];
  return e;
}

// Top-row loads of the marched vector for the pair.
template <typename T, typename ZT> struct VRaw2 {
  using T2 = typename V2<T>::t;
  T2 v0, v1;              // z, p_old, x, or b (SMOOTH0)
  ZT z0, z1;              // KP: z
  T2 c00, c10, c01, c11;  // PSMOOTH: coarse nodes (I, Jlo), (I+1, Jlo), (I, Jhi), (I+1, Jhi)
  double2 d1;             // SMOOTH0, float64 finest level: w / D of the pair
  T2 d20, d21;            // SMOOTH0, coarse levels: w / D per DOF
  double2 r0, r1, q0, q1;  // SMOOTH0 with the CG update: float64 r and q of the pair
};

// Node-row loads for the pair.
template <typename T> struct NRaw2 {
  using T2 = typename V2<T>::t;
  T2 b0, b1;
  T2 d20, d21;
  double2 d1;
};

// float64 dot partners of the pair (z.r, z.q), loaded one row ahead outside
// the lookahead ring: at 32 bytes per pair they would cost a ring slot's
// worth of registers.
struct DRaw2 {
  double2 rd0, rd1, qd0, qd1;
};

template <typename T, int SRC, int MODE, bool DOT, typename ZT> struct Sweep2 {
  using T2 = typename V2<T>::t;
  using S = Sweep<T, SRC, MODE, DOT, ZT>;
  using VR = VRaw2<T, ZT>;
  using ER = ERaw2<T, SRC>;
  using NR = NRaw2<T>;
  static constexpr bool SMOOTHING = S::SMOOTHING;
  // SMOOTH0 takes b and w/D of node row je from the previous step's top row.
  static constexpr bool NEEDS_B = S::NEEDS_B && MODE != MODE_SMOOTH0;
  // bf16 finest moduli run one row ahead of the elements.
  static constexpr bool E_AHEAD = SRC == SRC_FINEBF;

  // k: offset of node (i0, jj); i0 even.  lag (RESID): also load the
  // direction of the pending x step; (bf16 SMOOTH0 with the CG update): the
  // update is pending, load the last step's r.
  __device__ __forceinline__ static void load_v(const SweepParams<T>& a, long long k, int i0, int jj,
                                                VR& r, bool lag = false) {
    if constexpr (MODE == MODE_RESID) {
      ld_pair(a.v, k, r.v0, r.v1);
      if (lag) ld_pair(a.xdir, k, r.z0, r.z1);
    } else if constexpr (MODE == MODE_KP) {
      ld_pair(static_cast<const ZT*>(a.zkp), k, r.z0, r.z1);
      ld_pair(a.v, k, r.v0, r.v1);
    } else if constexpr (MODE == MODE_PSMOOTH) {
      ld_pair(a.v, k, r.v0, r.v1);
      // Node i0 sits on coarse column I = i0 / 2, node i1 halfway to I + 1;
      // row jj on coarse row jj / 2, or halfway between Jlo and Jhi when odd
      // (jj is uniform over the warp).
      const Grid gc = a.gc;
      const int I = i0 >> 1, Jlo = jj >> 1;
      const long long kc = gc.at(I, Jlo);
      r.c00 = a.zc[kc];
      r.c10 = a.zc[kc + 1];
      if (jj & 1) {
        r.c01 = a.zc[kc + gc.pitch];
        r.c11 = a.zc[kc + gc.pitch + 1];
      } else {
        r.c01 = r.c00;
        r.c11 = r.c10;
      }
    } else if constexpr (MODE == MODE_SMOOTH0) {
      if constexpr (SRC == SRC_FINEBF && DOT) {  // the CG update forms b from r and q
        ld_pair(lag ? a.r64_prev : static_cast<const double2*>(a.r64), k, r.r0, r.r1);
        ld_pair(a.q64, k, r.q0, r.q1);
      } else {
        ld_pair(a.b, k, r.v0, r.v1);
      }
      if constexpr (SRC == SRC_FINE64) r.d1 = reinterpret_cast<const double2*>(a.invd1)[k >> 1];
      else if constexpr (SRC != SRC_FINEBF) ld_pair(a.invd2, k, r.d20, r.d21);
    } else {
      ld_pair(a.v, k, r.v0, r.v1);
    }
  }

  // Marched values of the pair at row jj (SMOOTH0 on the bf16 level is formed
  // in the kernel, where the top-row D is known).
  __device__ __forceinline__ static void finish_v(const SweepParams<T>& a, const VR& r, int i0, int jj,
                                                  T beta, T2& o0, T2& o1, bool lag = false,
                                                  T alag = T(0)) {
    if constexpr (MODE == MODE_RESID) {
      o0 = r.v0;
      o1 = r.v1;
      if (lag) {  // x + alpha p: the iterate the pending step leads to
        o0 = mk2<T>(fma(alag, T(r.z0.x), o0.x), fma(alag, T(r.z0.y), o0.y));
        o1 = mk2<T>(fma(alag, T(r.z1.x), o1.x), fma(alag, T(r.z1.y), o1.y));
      }
    } else if constexpr (MODE == MODE_KP) {
      if constexpr (sizeof(T) == 8) {
        o0 = mk2<T>(to_f64(r.z0.x) + beta * r.v0.x, to_f64(r.z0.y) + beta * r.v0.y);
        o1 = mk2<T>(to_f64(r.z1.x) + beta * r.v1.x, to_f64(r.z1.y) + beta * r.v1.y);
      } else {
        o0 = mk2<T>(T(r.z0.x) + beta * r.v0.x, T(r.z0.y) + beta * r.v0.y);
        o1 = mk2<T>(T(r.z1.x) + beta * r.v1.x, T(r.z1.y) + beta * r.v1.y);
      }
    } else if constexpr (MODE == MODE_PSMOOTH) {
      const T h = T(0.5);
      const T2 cy0 = mk2<T>(h * (r.c00.x + r.c01.x), h * (r.c00.y + r.c01.y));
      const T2 cy1 = mk2<T>(h * (r.c10.x + r.c11.x), h * (r.c10.y + r.c11.y));
      o0 = a.g.valid(i0, jj) ? mk2<T>(r.v0.x + cy0.x, r.v0.y + cy0.y) : mk2<T>(T(0), T(0));
      o1 = a.g.valid(i0 + 1, jj)
               ? mk2<T>(r.v1.x + h * (cy0.x + cy1.x), r.v1.y + h * (cy0.y + cy1.y))
               : mk2<T>(T(0), T(0));
    } else if constexpr (MODE == MODE_SMOOTH0) {
      // w D^-1 is zero on clamped and ghost nodes, so no mask is needed.
      if constexpr (SRC == SRC_FINE64) {
        o0 = mk2<T>(T(r.d1.x) * r.v0.x, T(r.d1.x) * r.v0.y);
        o1 = mk2<T>(T(r.d1.y) * r.v1.x, T(r.d1.y) * r.v1.y);
      } else {
        o0 = mk2<T>(r.d20.x * r.v0.x, r.d20.y * r.v0.y);
        o1 = mk2<T>(r.d21.x * r.v1.x, r.d21.y * r.v1.y);
      }
    } else {
      o0 = r.v0;
      o1 = r.v1;
    }
  }

  // e: offset of element (i0, jj).
  __device__ __forceinline__ static void load_e(const SweepParams<T>& a, long long e, int i0, int jj,
                                                ER& r) {
    if constexpr (SRC == SRC_CFINE) {
      // Coarse elements i0 and i0 + 1 cover fine columns 2 i0 .. 2 i0 + 3
      // (8-byte aligned since i0 is even).  Element i0 + 1 = nx reads the
      // fine ghost columns, which are zero.
      if ((unsigned)i0 < (unsigned)a.g.nx && (unsigned)jj < (unsigned)a.g.ny) {
        const long long kf = a.gfine.at(2 * i0, 2 * jj);
        const uint2 lo = *reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(a.E) + kf);
        const uint2 hi = *reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(a.E) + kf +
                                                         a.gfine.pitch);
        r.lo[0] = *reinterpret_cast<const __nv_bfloat162*>(&lo.x);
        r.lo[1] = *reinterpret_cast<const __nv_bfloat162*>(&lo.y);
        r.hi[0] = *reinterpret_cast<const __nv_bfloat162*>(&hi.x);
        r.hi[1] = *reinterpret_cast<const __nv_bfloat162*>(&hi.y);
      } else {
        r.lo[0] = r.lo[1] = r.hi[0] = r.hi[1] = __floats2bfloat162_rn(0.f, 0.f);
      }
    } else if constexpr (SRC == SRC_FINE64) {
      const double2* p = static_cast<const double2*>(a.E) + 2 * e;
      r.k[0] = __ldg(p);
      r.k[1] = __ldg(p + 1);
      r.k[2] = __ldg(p + 2);
      r.k[3] = __ldg(p + 3);
    } else if constexpr (SRC == SRC_FINEBF) {
      const __nv_bfloat16* Eb = static_cast<const __nv_bfloat16*>(a.E);
      r.E = *reinterpret_cast<const __nv_bfloat162*>(Eb + e);
      // SMOOTH0 forms D at both columns of the top row, so every lane needs
      // the modulus of element i0 - 1 itself (lane 0 has no left lane).
      if constexpr (MODE == MODE_SMOOTH0) r.El = *reinterpret_cast<const __nv_bfloat162*>(Eb + e - 2);
    } else if constexpr (SRC == SRC_CMOM) {
      using T2c = typename V2<T>::t;
#pragma unroll
      for (int c = 0; c < NMOM; ++c) r.m[c] = *reinterpret_cast<const T2c*>(a.coef + c * a.cstride + e);
    } else {
      using T2c = typename V2<T>::t;
#pragma unroll
      for (int c = 0; c < NCOEF; ++c) r.A[c] = *reinterpret_cast<const T2c*>(a.coef + c * a.cstride + e);
    }
  }

  __device__ __forceinline__ static void load_n(const SweepParams<T>& a, long long k, NR& r) {
    if constexpr (NEEDS_B) ld_pair(a.b, k, r.b0, r.b1);
    if constexpr (SMOOTHING && MODE != MODE_SMOOTH0) {
      if constexpr (SRC == SRC_FINE64) r.d1 = reinterpret_cast<const double2*>(a.invd1)[k >> 1];
      else if constexpr (SRC == SRC_COARSE || SRC == SRC_CFINE || SRC == SRC_CMOM) ld_pair(a.invd2, k, r.d20, r.d21);
    }
  }

  __device__ __forceinline__ static void load_d(const SweepParams<T>& a, long long k, DRaw2& r) {
    ld_pair(a.rdot, k, r.rd0, r.rd1);
    if (a.qdot != nullptr) ld_pair(a.qdot, k, r.qd0, r.qd1);
  }

  // Strain-space forces of element w (0: i0, 1: i1) of the pair.
  __device__ __forceinline__ static Strain<T> core(const SweepParams<T>& a, const ER& er, int w,
                                                   const Strain<T>& s, T E) {
    if constexpr (SRC == SRC_FINEBF) {
      return fine_core<T>(s, E, a.kf);
    } else {
      T dummy;
      return S::core(a, pick(er, w), s, dummy);
    }
  }
};

// D^-1 w of the bf16 finest level at the pair of node row j from the moduli
// of element rows j - 1 (eb) and j (et): node i0 touches the elements i0 - 1
// (the left lane's second column) and i0, node i1 the elements i0 and i1.
// Lane 0's column i0 comes out wrong (no left lane); it is a halo column
// whose output is never written.
__device__ __forceinline__ void fbf_winv(float eb0, float eb1, float et0, float et1, float wdiag,
                                         float& w0, float& w1) {
  const float s0 = eb0 + et0, s1 = eb1 + et1;
  const float sl = __shfl_up_sync(0xffffffffu, s1, 1);
  w0 = __fdividef(wdiag, s0 + sl);
  w1 = __fdividef(wdiag, s0 + s1);
}
// The same with the moduli of element i0 - 1 given (ebl, etl): correct in
// every column, as needed where the values feed elements (SMOOTH0 top row).
__device__ __forceinline__ void fbf_winv_own(float ebl, float eb0, float eb1, float etl, float et0,
                                             float et1, float wdiag, float& w0, float& w1) {
  const float s0 = eb0 + et0, s1 = eb1 + et1;
  w0 = __fdividef(wdiag, s0 + (ebl + etl));
  w1 = __fdividef(wdiag, s0 + s1);
}

__device__ __forceinline__ float bf_lo(__nv_bfloat162 v) { return __low2float(v); }
__device__ __forceinline__ float bf_hi(__nv_bfloat162 v) { return __high2float(v); }

// One warp task of a two-column sweep: strip and chunk from the task index
// wg (all 32 lanes call it together).  Dot-product contributions accumulate
// into dot0 / dot1; the caller reduces them.
template <typename T, int SRC, int MODE, bool DOT, typename ZT, int PF>
__device__ __forceinline__ void sweep2_warp(const SweepParams<T>& a, int wg, int lane, double& dot0,
                                            double& dot1) {
  using T2 = typename V2<T>::t;
  using S2 = Sweep2<T, SRC, MODE, DOT, ZT>;
  using VR = typename S2::VR;
  using ER = typename S2::ER;
  using NR = typename S2::NR;
  constexpr bool FBF = SRC == SRC_FINEBF;
  constexpr bool FBF0 = FBF && MODE == MODE_SMOOTH0;
  // The bf16 pre-smoothing with DOT carries the CG update of the outer
  // iteration (Alg. 2): r -= alpha q at every node row it loads, b = float(r)
  // for the smoothing, and at the rows it owns the new r, its float32 copy
  // and |r|^2 (into dot0).  Without a pending update (the first iteration,
  // or one whose residual was just replaced) alpha is 0 and nothing is written.
  constexpr bool UPD = FBF0 && DOT;
  bool upd = false;
  double aupd = 0.0;
  if constexpr (UPD) {
    upd = a.sc->upd_pending != 0;
    aupd = upd ? a.sc->alpha : 0.0;
  }
  const int strip = wg % a.nstrips;
  const int chunk = wg / a.nstrips;
  T beta = T(0);
  if constexpr (MODE == MODE_KP) beta = T(a.sc->beta);
  bool vzero = false;
  if constexpr (MODE == MODE_RESID) vzero = a.zero_gate && a.sc->x_nonzero == 0;
  // Pending x step (x_lag): K p advances x at its owned nodes, the residual
  // replacement works on x + alpha p.
  bool lag = false;
  T alag = T(0);
  if constexpr (MODE == MODE_KP) {
    lag = a.sc->x_lag != 0;
    alag = T(a.sc->alpha);
  }
  if constexpr (MODE == MODE_RESID) {
    if (a.xlag && a.sc != nullptr && a.sc->x_lag != 0) {
      lag = true;
      alag = T(a.sc->alpha);
    }
  }
  if constexpr (UPD) lag = upd;  // read the last step's r

  constexpr int STRIDE = MODE == MODE_RESTRICT ? SWEEP2_RSTRIDE : SWEEP2_STRIDE;
  const Grid g = a.g;
  const int i0 = strip * STRIDE - 2 + 2 * lane;
  const bool own0 = lane >= 1 && i0 >= 0 && i0 <= g.nx;
  const bool own1 = lane <= 30 && i0 + 1 >= 0 && i0 + 1 <= g.nx;

  if (vzero) {
    // Residual of a zero iterate: r = b on the free DOFs, no operator needed.
    if (chunk < a.nchunks) {
      const int r0 = chunk * a.H, r1 = min(r0 + a.H - 1, g.ny);
      for (int j = r0; j <= r1; ++j) {
        const long long k = g.at(i0, j);
        T2 b0, b1;
        ld_pair(a.b, k, b0, b1);
        const T2 zero = mk2<T>(T(0), T(0));
        const T2 q0 = own0 && !g.is_fixed(i0, j) ? b0 : zero;
        const T2 q1 = own1 && !g.is_fixed(i0 + 1, j) ? b1 : zero;
        st_pair(a.out, k, q0, q1, own0, own1);
        if (a.out32 != nullptr)
          st_pair(a.out32, k, make_float2(float(q0.x), float(q0.y)), make_float2(float(q1.x), float(q1.y)),
                  own0, own1);
        dot0 += double(q0.x) * double(q0.x) + double(q0.y) * double(q0.y) +
                double(q1.x) * double(q1.x) + double(q1.y) * double(q1.y);
      }
    }
  } else if (chunk < a.nchunks) {
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
    const bool cfix0 = ((g.fixed & 2u) && i0 == 0) || ((g.fixed & 4u) && i0 == g.nx);
    const bool cfix1 = ((g.fixed & 2u) && i0 + 1 == 0) || ((g.fixed & 4u) && i0 + 1 == g.nx);
    const long long pitch = g.pitch;

    struct Pack {
      VR vt;
      ER e;
      NR n;
    };
    // Step je: node row je + 1, element row je (je + 1 for the bf16 moduli),
    // node row je.
    auto load_pack = [&](Pack& pk, int je, long long ke) {
      S2::load_v(a, ke + pitch, i0, je + 1, pk.vt, lag);
      if constexpr (S2::E_AHEAD) S2::load_e(a, ke + pitch, i0, je + 1, pk.e);
      else S2::load_e(a, ke, i0, je, pk.e);
      S2::load_n(a, ke, pk.n);
    };

    // Right-hand side of a loaded node row (the float32 r of the V-cycle);
    // with UPD, the CG update of that row, written back where `owned`.
    auto take_b = [&](const VR& r, long long kk, bool owned, T2& b0, T2& b1) {
      if constexpr (UPD) {
        const double2 n0 = make_double2(fma(-aupd, r.q0.x, r.r0.x), fma(-aupd, r.q0.y, r.r0.y));
        const double2 n1 = make_double2(fma(-aupd, r.q1.x, r.r1.x), fma(-aupd, r.q1.y, r.r1.y));
        b0 = make_float2(d2f_rn(n0.x), d2f_rn(n0.y));
        b1 = make_float2(d2f_rn(n1.x), d2f_rn(n1.y));
        if (upd && owned) {  // uniform over the warp
          st_pair(a.r64, kk, n0, n1, own0, own1);
          st_pair(a.out32, kk, b0, b1, own0, own1);
          if (own0) dot0 = fma(n0.x, n0.x, fma(n0.y, n0.y, dot0));
          if (own1) dot0 = fma(n1.x, n1.x, fma(n1.y, n1.y, dot0));
        }
      } else {
        (void)kk;
        (void)owned;
        b0 = r.v0;
        b1 = r.v1;
      }
    };

    const long long k0 = g.at(i0, je0);
    // bf16 moduli of the current element row (and of the row below for D);
    // ecl, epl: element i0 - 1 (SMOOTH0).
    float ec0 = 0.f, ec1 = 0.f, ep0 = 0.f, ep1 = 0.f, ecl = 0.f, epl = 0.f;
    if constexpr (FBF) {
      ER e;
      S2::load_e(a, k0, i0, je0, e);
      ec0 = bf_lo(e.E);
      ec1 = bf_hi(e.E);
      if constexpr (FBF0) {
        ecl = bf_hi(e.El);
        if (je0 >= 0) {
          S2::load_e(a, k0 - pitch, i0, je0 - 1, e);
          ep0 = bf_lo(e.E);
          ep1 = bf_hi(e.E);
          epl = bf_hi(e.El);
        }
      }
    }
    // SMOOTH0: right-hand side and w/D of node row je carried from the
    // previous step's top row.
    T2 bc0 = mk2<T>(T(0), T(0)), bc1 = bc0, wc0 = bc0, wc1 = bc0;
    // Marched values of the first row.
    T2 vb0, vb1;
    {
      VR r0;
      S2::load_v(a, k0, i0, je0, r0, lag);
      T2 b0r = mk2<T>(T(0), T(0)), b1r = b0r;
      if constexpr (MODE == MODE_SMOOTH0) take_b(r0, k0, false, b0r, b1r);  // row of the chunk below
      if constexpr (FBF0) {
        float w0, w1;
        fbf_winv_own(epl, ep0, ep1, ecl, ec0, ec1, float(a.wdiag), w0, w1);
        const bool rowok = je0 >= 0 && je0 <= g.ny &&
                           !(((g.fixed & 1u) && je0 == 0) || ((g.fixed & 8u) && je0 == g.ny));
        const bool a0 = rowok && i0 >= 0 && i0 <= g.nx && !cfix0;
        const bool a1 = rowok && i0 + 1 >= 0 && i0 + 1 <= g.nx && !cfix1;
        wc0 = a0 ? mk2<T>(w0, w0) : mk2<T>(T(0), T(0));
        wc1 = a1 ? mk2<T>(w1, w1) : mk2<T>(T(0), T(0));
        vb0 = mk2<T>(wc0.x * b0r.x, wc0.y * b0r.y);
        vb1 = mk2<T>(wc1.x * b1r.x, wc1.y * b1r.y);
      } else {
        S2::finish_v(a, r0, i0, je0, beta, vb0, vb1, lag, alag);
      }
      if constexpr (MODE == MODE_SMOOTH0) {
        bc0 = b0r;
        bc1 = b1r;
        if constexpr (SRC == SRC_FINE64) {
          wc0 = mk2<T>(T(r0.d1.x), T(r0.d1.x));
          wc1 = mk2<T>(T(r0.d1.y), T(r0.d1.y));
        } else if constexpr (!FBF) {
          wc0 = r0.d20;
          wc1 = r0.d21;
        }
      }
    }
    T2 vb2 = shfl_down2(vb0);
    T2 ac0 = sub2(vb1, vb0), ac1 = sub2(vb2, vb1);  // bottom edges of the current element row
    const T2 zero2 = mk2<T>(T(0), T(0));
    T2 gbp0 = zero2, gbp1 = zero2, gvp0 = zero2, gvp1 = zero2;
    T2 racc = zero2;  // RESTRICT: partial coarse row
    if constexpr (FBF && !FBF0) {
      ep0 = 0.f;
      ep1 = 0.f;
    }

    Pack ring[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u)
      if (je0 + u <= je1) load_pack(ring[u], je0 + u, k0 + u * pitch);
    // Dot partners of node row je + 1 (dnext) and je (dcur).

    long long k = k0;  // offset of node / element (i0, je)
    for (int jb = je0; jb <= je1; jb += PF) {
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int je = jb + u;
        if (je > je1) break;
        const Pack cur = ring[u];
        if (je + PF <= je1) load_pack(ring[u], je + PF, k + PF * pitch);
        if constexpr (MODE == MODE_KP) {
          // Pending x step at the top row (owned rows only): x += alpha p_old.
          // Done at once, so that x occupies registers only briefly; other
          // warps cover the load with FP64 work.
          if (lag && je + 1 <= je1) {  // uniform over the warp
            T2 x0, x1;
            ld_pair(a.xvec, k + pitch, x0, x1);
            x0 = mk2<T>(fma(alag, cur.vt.v0.x, x0.x), fma(alag, cur.vt.v0.y, x0.y));
            x1 = mk2<T>(fma(alag, cur.vt.v1.x, x1.x), fma(alag, cur.vt.v1.y, x1.y));
            st_pair(a.xvec, k + pitch, x0, x1, own0, own1);
          }
        }
        DRaw2 dcur;
        if constexpr (DOT && !UPD) {
          if (je > je0) S2::load_d(a, k, dcur);
          // The float64 operands two rows up go to L2 now, so that their loads
          // there find them on chip.
          if (je + 2 <= je1) {
            prefetch_l2(a.rdot + k + 2 * pitch);
            if (a.qdot != nullptr) prefetch_l2(a.qdot + k + 2 * pitch);
          }
        }
        if constexpr (UPD) {
          if (je + PF + 2 <= je1) {  // the last step's r and q, rows beyond the ring
            prefetch_l2((lag ? a.r64_prev : a.r64) + k + (PF + 2) * pitch);
            prefetch_l2(a.q64 + k + (PF + 2) * pitch);
          }
        }
        if constexpr (FBF && MODE == MODE_RESTRICT) {
          if (je + PF + 2 <= je1) {  // marched vector, b and moduli beyond the ring
            const long long kp = k + (PF + 2) * pitch;
            prefetch_l2(a.v + kp);
            prefetch_l2(a.b + kp);
            prefetch_l2(static_cast<const __nv_bfloat16*>(a.E) + kp);
          }
        }

        // ---- top row je + 1 ----
        T2 vt0, vt1;
        float en0 = 0.f, en1 = 0.f, enl = 0.f;  // bf16 moduli of element row je + 1
        T2 wt0 = zero2, wt1 = zero2;
        T2 btop0 = zero2, btop1 = zero2;  // SMOOTH0: right-hand side of row je + 1
        if constexpr (MODE == MODE_SMOOTH0) take_b(cur.vt, k + pitch, je + 1 <= je1, btop0, btop1);
        if constexpr (FBF) {
          en0 = bf_lo(cur.e.E);
          en1 = bf_hi(cur.e.E);
        }
        if constexpr (FBF0) {
          enl = bf_hi(cur.e.El);
          float w0, w1;
          fbf_winv_own(ecl, ec0, ec1, enl, en0, en1, float(a.wdiag), w0, w1);
          const int jt = je + 1;
          const bool rowok =
              jt <= g.ny && !(((g.fixed & 1u) && jt == 0) || ((g.fixed & 8u) && jt == g.ny));
          const bool a0 = rowok && i0 >= 0 && i0 <= g.nx && !cfix0;
          const bool a1 = rowok && i0 + 1 >= 0 && i0 + 1 <= g.nx && !cfix1;
          wt0 = a0 ? mk2<T>(w0, w0) : zero2;
          wt1 = a1 ? mk2<T>(w1, w1) : zero2;
          vt0 = mul2(wt0, btop0);
          vt1 = mul2(wt1, btop1);
        } else {
          S2::finish_v(a, cur.vt, i0, je + 1, beta, vt0, vt1, lag, alag);
        }

        const T2 vt2 = shfl_down2(vt0);  // lane 31: its own value, used only for halo output
        const T2 bt0 = sub2(vt1, vt0), bt1 = sub2(vt2, vt1);  // top edges
        const T2 dl0 = sub2(vt0, vb0), dl1 = sub2(vt1, vb1);  // vertical edges at i0, i1
        T2 dl2;                                               // vertical edge at i0 + 2
        if constexpr (sizeof(T) == 8) dl2 = shfl_down2(dl0);  // a shuffle is cheaper than FP64
        else dl2 = sub2(vt2, vb2);
        // Strain coordinates as component pairs: (c1, d1) = a + b,
        // (c3, d3) = b - a, (c2, d2) = dl + dr, s = c2 + d1.
        Strain<T> w0, w1;
        {
          const T2 cd1 = add2(ac0, bt0), cd3 = sub2(bt0, ac0), cd2 = add2(dl0, dl1);
          w0.c1 = cd1.x;
          w0.c3 = cd3.x;
          w0.d3 = cd3.y;
          w0.d2 = cd2.y;
          w0.s = cd2.x + cd1.y;
        }
        {
          const T2 cd1 = add2(ac1, bt1), cd3 = sub2(bt1, ac1), cd2 = add2(dl1, dl2);
          w1.c1 = cd1.x;
          w1.c3 = cd3.x;
          w1.d3 = cd3.y;
          w1.d2 = cd2.y;
          w1.s = cd2.x + cd1.y;
        }
        const ER& ecur_raw = cur.e;  // element row je for every source but the bf16 moduli
        const Strain<T> t0 = S2::core(a, ecur_raw, 0, w0, T(ec0));
        const Strain<T> t1 = S2::core(a, ecur_raw, 1, w1, T(ec1));
        // ---- edge forces and node row je ----
        const T2 p0 = mk2<T>(t0.c1, t0.s), m0p = mk2<T>(t0.c3, t0.d3);
        const T2 p1 = mk2<T>(t1.c1, t1.s), m1p = mk2<T>(t1.c3, t1.d3);
        const T2 ga0 = sub2(p0, m0p), gb0 = add2(p0, m0p);
        const T2 ga1 = sub2(p1, m1p), gb1 = add2(p1, m1p);
        const T2 gs0 = mk2<T>(t0.s, t0.d2), gs1 = mk2<T>(t1.s, t1.d2);
        const T2 gh0 = add2(ga0, gbp0);  // horizontal edge i0 -> i1 of row je
        const T2 gh1 = add2(ga1, gbp1);  // i1 -> i0 + 2
        const T2 ghl = shfl_up2(gh1);    // i0 - 1 -> i0
        const T2 gv0 = add2(gs0, shfl_up2(gs1));  // vertical edge at i0, rows je -> je + 1
        const T2 gv1 = add2(gs0, gs1);            // at i1
        const T2 kv0 = add2(sub2(ghl, gh0), sub2(gvp0, gv0));
        const T2 kv1 = add2(sub2(gh0, gh1), sub2(gvp1, gv1));

        bool inrow = je > je0;
        if constexpr (MODE == MODE_RESTRICT) inrow = inrow && je <= g.ny;
        const bool rfix = ((g.fixed & 1u) && je == 0) || ((g.fixed & 8u) && je == g.ny);
        const bool inb0 = inrow && own0, inb1 = inrow && own1;
        const bool act0 = inb0 && !cfix0 && !rfix, act1 = inb1 && !cfix1 && !rfix;

        if constexpr (MODE == MODE_APPLY) {
          if constexpr (sizeof(T) == 4) {  // mask by multiplication (FMA pipe, values finite)
            const T m0 = act0 ? T(1) : T(0), m1 = act1 ? T(1) : T(0);
            st_pair(a.out, k, mk2<T>(kv0.x * m0, kv0.y * m0), mk2<T>(kv1.x * m1, kv1.y * m1), inb0, inb1);
          } else {
            st_pair(a.out, k, act0 ? kv0 : zero2, act1 ? kv1 : zero2, inb0, inb1);
          }
        } else if constexpr (MODE == MODE_RESID) {
          const T2 r0 = act0 ? sub2(cur.n.b0, kv0) : zero2;
          const T2 r1 = act1 ? sub2(cur.n.b1, kv1) : zero2;
          st_pair(a.out, k, r0, r1, inb0, inb1);
          if (a.out32 != nullptr)
            st_pair(a.out32, k, make_float2(float(r0.x), float(r0.y)),
                    make_float2(float(r1.x), float(r1.y)), inb0, inb1);
          dot0 = fma(double(r0.x), double(r0.x), fma(double(r0.y), double(r0.y), dot0));
          dot0 = fma(double(r1.x), double(r1.x), fma(double(r1.y), double(r1.y), dot0));
        } else if constexpr (MODE == MODE_KP) {
          const T2 q0 = act0 ? kv0 : zero2, q1 = act1 ? kv1 : zero2;
          st_pair(a.p_out, k, vb0, vb1, inb0, inb1);
          st_pair(a.out, k, q0, q1, inb0, inb1);
          if (inb0) dot0 = fma(double(vb0.x), double(q0.x), fma(double(vb0.y), double(q0.y), dot0));
          if (inb1) dot0 = fma(double(vb1.x), double(q1.x), fma(double(vb1.y), double(q1.y), dot0));
        } else if constexpr (S2::SMOOTHING) {
          T2 b0, b1, d0, d1;
          if constexpr (MODE == MODE_SMOOTH0) {
            b0 = bc0;
            b1 = bc1;
            d0 = wc0;
            d1 = wc1;
          } else {
            b0 = cur.n.b0;
            b1 = cur.n.b1;
            if constexpr (SRC == SRC_FINE64) {
              d0 = mk2<T>(T(cur.n.d1.x), T(cur.n.d1.x));
              d1 = mk2<T>(T(cur.n.d1.y), T(cur.n.d1.y));
            } else if constexpr (FBF) {
              // D from the moduli is zero on ghost nodes: mask w / D itself.
              float w0f, w1f;
              fbf_winv(ep0, ep1, ec0, ec1, float(a.wdiag), w0f, w1f);
              w0f = act0 ? w0f : 0.f;
              w1f = act1 ? w1f : 0.f;
              d0 = mk2<T>(w0f, w0f);
              d1 = mk2<T>(w1f, w1f);
            } else {
              d0 = cur.n.d20;
              d1 = cur.n.d21;
            }
          }
          // w / D, the marched v and b all vanish on clamped and ghost nodes,
          // so z does too without a select.
          const T2 z0 = fma2(d0, sub2(b0, kv0), vb0);
          const T2 z1 = fma2(d1, sub2(b1, kv1), vb1);
          st_pair(a.out, k, z0, z1, inb0, inb1);
          if constexpr (DOT && !UPD) {
            // Inactive nodes contribute 0 (z and r vanish there).
            if (inb0) {
              const double zx = to_f64(z0.x), zy = to_f64(z0.y);
              dot0 = fma(zx, dcur.rd0.x, fma(zy, dcur.rd0.y, dot0));
              if (a.qdot != nullptr) dot1 = fma(zx, dcur.qd0.x, fma(zy, dcur.qd0.y, dot1));
            }
            if (inb1) {
              const double zx = to_f64(z1.x), zy = to_f64(z1.y);
              dot0 = fma(zx, dcur.rd1.x, fma(zy, dcur.rd1.y, dot0));
              if (a.qdot != nullptr) dot1 = fma(zx, dcur.qd1.x, fma(zy, dcur.qd1.y, dot1));
            }
          }
        } else if constexpr (MODE == MODE_RESTRICT) {
          const T m0 = act0 ? T(1) : T(0), m1 = act1 ? T(1) : T(0);  // multiplicative masks
          const T2 r0 = mul2(sub2(cur.n.b0, kv0), mk2<T>(m0, m0));
          const T2 r1 = mul2(sub2(cur.n.b1, kv1), mk2<T>(m1, m1));
          // Horizontal full weighting (1/2, 1, 1/2) onto coarse column
          // I = i0 / 2 (lanes 1..30), then vertical accumulation along the
          // march over fine rows 2J - 1, 2J, 2J + 1.
          const T2 rl = shfl_up2(r1);
          const T2 h = mk2<T>(r0.x + T(0.5) * (r1.x + rl.x), r0.y + T(0.5) * (r1.y + rl.y));
          if (je > je0) {
            if (je & 1) {
              const int Jlo = (je - 1) / 2;
              const T2 val = mk2<T>(racc.x + T(0.5) * h.x, racc.y + T(0.5) * h.y);
              const int I = i0 >> 1;
              if (lane >= 1 && lane <= 30 && Jlo >= Jb && Jlo <= Je && I >= 0 && I <= a.gc.nx) {
                a.bc[a.gc.at(I, Jlo)] = a.gc.is_fixed(I, Jlo) ? zero2 : val;
              }
              racc = mk2<T>(T(0.5) * h.x, T(0.5) * h.y);
            } else {
              racc = add2(racc, h);
            }
          }
        }
        if constexpr (MODE == MODE_SMOOTH0) {
          bc0 = btop0;
          bc1 = btop1;
          if constexpr (FBF0) {
            wc0 = wt0;
            wc1 = wt1;
          } else if constexpr (SRC == SRC_FINE64) {
            wc0 = mk2<T>(T(cur.vt.d1.x), T(cur.vt.d1.x));
            wc1 = mk2<T>(T(cur.vt.d1.y), T(cur.vt.d1.y));
          } else {
            wc0 = cur.vt.d20;
            wc1 = cur.vt.d21;
          }
        }
        if constexpr (FBF) {
          ep0 = ec0;
          ep1 = ec1;
          ec0 = en0;
          ec1 = en1;
          ecl = enl;
        }
        ac0 = bt0;
        ac1 = bt1;
        gbp0 = gb0;
        gbp1 = gb1;
        gvp0 = gv0;
        gvp1 = gv1;
        vb0 = vt0;
        vb1 = vt1;
        vb2 = vt2;
        k += pitch;
      }
    }
  }
}

// Two resident blocks per SM (at most 128 registers per thread): one full
// wave is then 16 warps per SM, which the launch shapes assume.
template <typename T, int SRC, int MODE, bool DOT, typename ZT, int PF>
__global__ void __launch_bounds__(SWEEP_NT, 2) sweep2_kernel(const SweepParams<T> a) {
  constexpr bool REDUCE = DOT || MODE == MODE_RESID || MODE == MODE_KP;
  pdl_wait();
  if (a.sc != nullptr && a.gate) {
    if (a.sc->done != RUNNING) return;  // uniform over the grid
    if (a.replace_gate && (a.sc->rr_every <= 0 || (a.sc->iter % a.sc->rr_every) != 0)) return;
  }
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (SWEEP_NT / 32) + (threadIdx.x >> 5);
  double dot0 = 0.0, dot1 = 0.0;
  sweep2_warp<T, SRC, MODE, DOT, ZT, PF>(a, wg, lane, dot0, dot1);
  if constexpr (REDUCE) {
    block_reduce_finish<SWEEP_NT>(dot0, dot1, a.partials, a.ticket, a.sc, a.finish, a.out_value,
                                  a.tag);
  }
}

}  // namespace mto
