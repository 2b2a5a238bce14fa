// Matrix-free stencil sweeps of the V-cycle and the outer CG operator.
//
// One warp owns a strip of node columns and a chunk of rows.  Lane L holds
// node column i and marches upwards one element row per step: it loads the
// node values of the new top row (the right neighbour's come by shuffle),
// computes the element (i, je) to its right once, and completes node row je
// from the four element forces that touch it (two of them arrive from the
// left lane by shuffle, two were carried from the previous step).  Lanes
// 1..31 of a warp own complete columns; lane 0 overlaps the previous strip.
// Every element is therefore evaluated once per strip (32/31 overall), every
// node value is read once from memory, and no shared memory or atomics are
// needed.
//
// Modes (all masked by the clamped edges; ghost nodes are zero by layout):
//   APPLY    out = K v
//   RESID    out = b - K v,                       dot |out|^2
//   KP       p = z + beta p_old, q = K p,          dot p.q      (Alg. 2)
//   SMOOTH   out = v + w D^-1 (b - K v)                          (Sec. 2.3)
//   PSMOOTH  v' = v + P zc (Alg. 1 correction), out = v' + w D^-1 (b - K v')
//   RESTRICT bc = P^T (b - K v) on the next coarser grid        (Alg. 1)
// SMOOTH/PSMOOTH optionally accumulate z.r (and z.q for the flexible beta).
#pragma once

#include "mto_common.cuh"

namespace mto {

constexpr int SWEEP_NT = 256;

enum Src { SRC_FINE64 = 0, SRC_FINEBF = 1, SRC_COARSE = 2 };
enum Mode { MODE_APPLY = 0, MODE_RESID, MODE_KP, MODE_SMOOTH, MODE_PSMOOTH, MODE_RESTRICT };

template <typename T> struct SweepParams {
  using T2 = typename V2<T>::t;
  Grid g;   // this level
  Grid gc;  // next coarser level (PSMOOTH source, RESTRICT target)
  int nstrips, nchunks, H;
  int gate;          // 1: skip the launch once the PCG has stopped (sc->done)
  int replace_gate;  // RESID as residual replacement: run only when iter % rr_every == 0
  const T2* v;       // marched vector (z, x or p_old)
  const T2* zc;      // PSMOOTH: coarse correction
  const void* zkp;   // KP: z (double2 or float2)
  T2* p_out;         // KP: new search direction
  const T2* b;       // right-hand side (SMOOTH, PSMOOTH, RESTRICT, RESID)
  T2* out;           // output vector (APPLY, RESID, KP: q, SMOOTH, PSMOOTH)
  T2* bc;            // RESTRICT: coarse right-hand side
  const void* E;     // fine moduli (double or bf16), padded element layout
  const T* coef;     // coarse element matrices, NCOEF arrays of g.size()
  long long cstride;
  FineConst<T> kf;
  const double* invd1;  // float64 fine level: w / D per node
  const T2* invd2;      // coarse levels: w / D per DOF
  T wdiag;              // float32 fine level: w / (KE_00 at E = 1); D = sum of 4 moduli
  const double2* rdot;  // dot partner for z.r
  const double2* qdot;  // dot partner for z.q (flexible beta), may be null
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

__device__ __forceinline__ float load_e(const void* E, long long k, float) {
  return __bfloat162float(static_cast<const __nv_bfloat16*>(E)[k]);
}
__device__ __forceinline__ double load_e(const void* E, long long k, double) {
  return __ldg(static_cast<const double*>(E) + k);
}

template <typename T, int SRC, int MODE, bool DOT, typename ZT>
__global__ void __launch_bounds__(SWEEP_NT) sweep_kernel(const SweepParams<T> a) {
  using T2 = typename V2<T>::t;
  constexpr bool REDUCE = DOT || MODE == MODE_RESID || MODE == MODE_KP;
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

  if (chunk < a.nchunks) {
    constexpr int STRIDE = MODE == MODE_RESTRICT ? 30 : 31;
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

    // Value of the marched vector at node (ii, jj).
    auto load_v = [&](int ii, int jj) -> T2 {
      const long long k = g.at(ii, jj);
      if constexpr (MODE == MODE_KP) {
        const ZT zz = static_cast<const ZT*>(a.zkp)[k];
        const T2 pp = a.v[k];
        return mk2<T>(T(zz.x) + beta * pp.x, T(zz.y) + beta * pp.y);
      } else if constexpr (MODE == MODE_PSMOOTH) {
        if (!g.valid(ii, jj)) return mk2<T>(T(0), T(0));
        const T2 zz = a.v[k];
        const int I0 = ii >> 1, J0 = jj >> 1;
        const T wx0 = (ii & 1) ? T(0.5) : T(1), wx1 = (ii & 1) ? T(0.5) : T(0);
        const T wy0 = (jj & 1) ? T(0.5) : T(1), wy1 = (jj & 1) ? T(0.5) : T(0);
        const Grid gc = a.gc;
        const T2 c00 = a.zc[gc.at(I0, J0)], c10 = a.zc[gc.at(I0 + 1, J0)];
        const T2 c01 = a.zc[gc.at(I0, J0 + 1)], c11 = a.zc[gc.at(I0 + 1, J0 + 1)];
        const T ix = wy0 * (wx0 * c00.x + wx1 * c10.x) + wy1 * (wx0 * c01.x + wx1 * c11.x);
        const T iy = wy0 * (wx0 * c00.y + wx1 * c10.y) + wy1 * (wx0 * c01.y + wx1 * c11.y);
        return mk2<T>(zz.x + ix, zz.y + iy);
      } else {
        return a.v[k];
      }
    };

    T2 vb = load_v(i, je0);
    T2 vbr = shfl_down2(vb);
    if (lane == 31) vbr = load_v(i + 1, je0);
    T2 cTL = mk2<T>(T(0), T(0)), cTR = cTL;
    T Eprev = T(0);
    T2 racc = mk2<T>(T(0), T(0));  // RESTRICT: partial coarse row

    for (int je = je0; je <= je1; ++je) {
      T2 vt = load_v(i, je + 1);
      T2 vtr = shfl_down2(vt);
      if (lane == 31) vtr = load_v(i + 1, je + 1);
      const long long e = g.at(i, je);
      const Strain<T> w = strain_coords<T>(vb, vbr, vtr, vt);
      Strain<T> t;
      T Ecur = T(0);
      if constexpr (SRC == SRC_COARSE) {
        T A[NCOEF];
#pragma unroll
        for (int k = 0; k < NCOEF; ++k) A[k] = a.coef[k * a.cstride + e];
        t = coarse_core<T>(w, A);
      } else {
        Ecur = load_e(a.E, e, T(0));
        t = fine_core<T>(w, Ecur, a.kf);
      }
      T2 fBL, fBR, fTR, fTL;
      strain_forces<T>(t, fBL, fBR, fTR, fTL);
      // Node (i, je): own element's BL force, left element's BR force (shuffle),
      // and the TL / TR forces of the element row below (carried).
      const T2 sl = shfl_up2(add2(cTR, fBR));
      const T2 kv = add2(add2(cTL, fBL), sl);
      T eol = T(0), eo = T(0);
      if constexpr (SRC == SRC_FINEBF && (MODE == MODE_SMOOTH || MODE == MODE_PSMOOTH)) {
        eo = Eprev + Ecur;
        eol = __shfl_up_sync(0xffffffffu, eo, 1);
        Eprev = Ecur;
      }
      const bool emit = je > je0 && lane >= 1;
      const bool inb = emit && g.valid(i, je);
      const bool act = inb && !g.is_fixed(i, je);
      const long long k = e;  // node (i, je) shares the element's offset
      if constexpr (MODE == MODE_APPLY) {
        if (inb) a.out[k] = act ? kv : mk2<T>(T(0), T(0));
      } else if constexpr (MODE == MODE_RESID) {
        T2 r = mk2<T>(T(0), T(0));
        if (act) r = sub2(a.b[k], kv);
        if (inb) a.out[k] = r;
        dot0 += double(r.x) * double(r.x) + double(r.y) * double(r.y);
      } else if constexpr (MODE == MODE_KP) {
        const T2 q = act ? kv : mk2<T>(T(0), T(0));
        if (inb) {
          a.p_out[k] = vb;
          a.out[k] = q;
        }
        dot0 += double(vb.x) * double(q.x) + double(vb.y) * double(q.y);
      } else if constexpr (MODE == MODE_SMOOTH || MODE == MODE_PSMOOTH) {
        T2 zn = mk2<T>(T(0), T(0));
        if (act) {
          const T2 res = sub2(a.b[k], kv);
          T dx, dy;
          if constexpr (SRC == SRC_FINE64) {
            dx = dy = T(a.invd1[k]);
          } else if constexpr (SRC == SRC_FINEBF) {
            dx = dy = a.wdiag / (eo + eol);
          } else {
            const T2 d = a.invd2[k];
            dx = d.x;
            dy = d.y;
          }
          zn = mk2<T>(vb.x + dx * res.x, vb.y + dy * res.y);
        }
        if (inb) a.out[k] = zn;
        if constexpr (DOT) {
          if (act) {
            const double2 rr = a.rdot[k];
            dot0 += double(zn.x) * rr.x + double(zn.y) * rr.y;
            if (a.qdot != nullptr) {
              const double2 qq = a.qdot[k];
              dot1 += double(zn.x) * qq.x + double(zn.y) * qq.y;
            }
          }
        }
      } else if constexpr (MODE == MODE_RESTRICT) {
        T2 r = mk2<T>(T(0), T(0));
        if (act) r = sub2(a.b[k], kv);
        // Horizontal full weighting (1/2, 1, 1/2) by shuffles, then vertical
        // accumulation along the march.
        const T2 ru = shfl_up2(r), rd = shfl_down2(r);
        const T2 h = mk2<T>(r.x + T(0.5) * (ru.x + rd.x), r.y + T(0.5) * (ru.y + rd.y));
        if (je > je0) {
          if (je & 1) {
            const int Jlo = (je - 1) / 2;
            const T2 val = mk2<T>(racc.x + T(0.5) * h.x, racc.y + T(0.5) * h.y);
            const bool producer = (lane & 1) == 0 && lane >= 2 && lane <= 30;
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
      cTL = fTL;
      cTR = fTR;
      vb = vt;
      vbr = vtr;
    }
  }
  if constexpr (REDUCE) {
    block_reduce_finish<SWEEP_NT>(dot0, dot1, a.partials, a.ticket, a.sc, a.finish, a.out_value);
  }
}

}  // namespace mto
