// Two-stage marching sweeps of the float32 coarse levels (Alg. 1): the
// pre-smoothing with the residual and its restriction, and the prolongation
// with the post-smoothing, each as one marching pass over the level.
//
// A stage is a marching sweep of mto_sweep2.cuh.  Stage B runs one node row
// behind stage A on the values stage A has just produced, in registers: at
// step je stage A completes node row je, and stage B evaluates element row
// je - 1 and completes node row je - 1, reusing the element data (and the
// right-hand side, D^-1) that stage A loaded one step earlier.  The
// intermediate vector never goes to memory, and the two sweeps cost one
// launch and one pass over the level's data.
//
//   PRE2:  stage A = SMOOTH0 (z1: two damped-Jacobi sweeps from zero),
//          stage B = residual b - K z1 and its full-weighting restriction.
//   POST2: stage A = PSMOOTH (z2 = v + w D^-1 (b - K v), v = z + P z_c),
//          stage B = one more sweep z3 = z2 + w D^-1 (b - K z2).
//
// Each stage loses one column at each side of the warp (a value needs its
// neighbours of the stage before), so a warp of POST2 outputs 60 columns
// (lanes 1-30), one of PRE2 29 coarse columns (lanes 2-30), and stage A runs
// over more rows than the chunk; the halo work is recomputed by the
// neighbouring tasks.  One 256-thread block per SM: the two stages together
// hold about 240 registers per thread.
#pragma once

#include "mto_sweep2.cuh"

namespace mto {

constexpr int POST2_STRIDE = 60;  // output columns per warp
constexpr int PRE2_CSTRIDE = 29;  // output coarse columns per warp

// One element row of a marching sweep over a pair of columns per lane:
// marched values vb (node row jj; vb2 = the right neighbour's first column)
// and vt (row jj + 1), bottom edges ac and edge forces gbp, gvp carried from
// the element row below.  Returns K v at node row jj in kv and advances the
// carried state to the next row.
template <typename S2>
__device__ __forceinline__ void element_row2(const SweepParams<float>& a, const typename S2::ER& e,
                                             const float2& vb0, const float2& vb1, const float2& vb2,
                                             const float2& vt0, const float2& vt1, float2& ac0,
                                             float2& ac1, float2& gbp0, float2& gbp1, float2& gvp0,
                                             float2& gvp1, float2& kv0, float2& kv1) {
  using T = float;
  using T2 = float2;
  const T2 vt2 = shfl_down2(vt0);
  const T2 bt0 = sub2(vt1, vt0), bt1 = sub2(vt2, vt1);
  const T2 dl0 = sub2(vt0, vb0), dl1 = sub2(vt1, vb1), dl2 = sub2(vt2, vb2);
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
  const Strain<T> t0 = S2::core(a, e, 0, w0, T(0));
  const Strain<T> t1 = S2::core(a, e, 1, w1, T(0));
  const T2 p0 = mk2<T>(t0.c1, t0.s), m0p = mk2<T>(t0.c3, t0.d3);
  const T2 p1 = mk2<T>(t1.c1, t1.s), m1p = mk2<T>(t1.c3, t1.d3);
  const T2 ga0 = sub2(p0, m0p), gb0 = add2(p0, m0p);
  const T2 ga1 = sub2(p1, m1p), gb1 = add2(p1, m1p);
  const T2 gs0 = mk2<T>(t0.s, t0.d2), gs1 = mk2<T>(t1.s, t1.d2);
  const T2 gh0 = add2(ga0, gbp0), gh1 = add2(ga1, gbp1);
  const T2 ghl = shfl_up2(gh1);
  const T2 gv0 = add2(gs0, shfl_up2(gs1)), gv1 = add2(gs0, gs1);
  kv0 = add2(sub2(ghl, gh0), sub2(gvp0, gv0));
  kv1 = add2(sub2(gh0, gh1), sub2(gvp1, gv1));
  ac0 = bt0;
  ac1 = bt1;
  gbp0 = gb0;
  gbp1 = gb1;
  gvp0 = gv0;
  gvp1 = gv1;
}

template <int SRC, int PF>
__device__ __forceinline__ void post2_warp(const SweepParams<float>& a, int wg, int lane) {
  using T = float;
  using T2 = float2;
  using S2 = Sweep2<float, SRC, MODE_PSMOOTH, false, float2>;
  using VR = typename S2::VR;
  using ER = typename S2::ER;
  using NR = typename S2::NR;
  const int strip = wg % a.nstrips;
  const int chunk = wg / a.nstrips;
  if (chunk >= a.nchunks) return;
  const Grid g = a.g;
  const int i0 = strip * POST2_STRIDE - 2 + 2 * lane;
  const bool own0 = lane >= 1 && lane <= 30 && i0 >= 0 && i0 <= g.nx;
  const bool own1 = lane >= 1 && lane <= 30 && i0 + 1 >= 0 && i0 + 1 <= g.nx;
  const int r0 = chunk * a.H, r1 = min(r0 + a.H - 1, g.ny);
  const int je0 = max(r0 - 2, -1), je1 = r1 + 1;  // stage A's steps (rows of z2: je0 + 1 .. je1)
  const long long pitch = g.pitch;
  const T2 zero2 = make_float2(0.f, 0.f);

  struct Pack {
    VR vt;
    ER e;
    NR n;
  };
  auto load_pack = [&](Pack& pk, int je, long long ke) {
    S2::load_v(a, ke + pitch, i0, je + 1, pk.vt);
    S2::load_e(a, ke, i0, je, pk.e);
    S2::load_n(a, ke, pk.n);
  };

  // Stage A: marched values of the first row.
  const long long k0 = g.at(i0, je0);
  T2 vb0, vb1;
  {
    VR r;
    S2::load_v(a, k0, i0, je0, r);
    S2::finish_v(a, r, i0, je0, T(0), vb0, vb1);
  }
  T2 vb2 = shfl_down2(vb0);
  T2 ac0 = sub2(vb1, vb0), ac1 = sub2(vb2, vb1);
  T2 gbp0 = zero2, gbp1 = zero2, gvp0 = zero2, gvp1 = zero2;
  // Stage B: z2 of its bottom node row (zero below the first row of z2,
  // which is also the value of the ghost row -1), its edges and forces, and
  // the element and node data of that row from stage A's last step.
  T2 zb0 = zero2, zb1 = zero2, zb2 = zero2;
  T2 bac0 = zero2, bac1 = zero2, bgbp0 = zero2, bgbp1 = zero2, bgvp0 = zero2, bgvp1 = zero2;
  ER eprev{};
  NR nprev{};

  Pack ring[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u)
    if (je0 + u <= je1) load_pack(ring[u], je0 + u, k0 + u * pitch);

  long long k = k0;  // node (i0, je)
  for (int jb = je0; jb <= je1; jb += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int je = jb + u;
      if (je > je1) break;
      const Pack cur = ring[u];
      if (je + PF <= je1) load_pack(ring[u], je + PF, k + PF * pitch);

      // ---- stage A: z2 at node row je ----
      T2 vt0, vt1;
      S2::finish_v(a, cur.vt, i0, je + 1, T(0), vt0, vt1);
      T2 kv0, kv1;
      element_row2<S2>(a, cur.e, vb0, vb1, vb2, vt0, vt1, ac0, ac1, gbp0, gbp1, gvp0, gvp1, kv0, kv1);
      // D^-1 and v vanish on clamped and ghost nodes, so z2 does too.  The
      // first step has no row below: its z2 is never used.
      const bool valid = je > je0;
      const T2 z20 = valid ? fma2(cur.n.d20, sub2(cur.n.b0, kv0), vb0) : zero2;
      const T2 z21 = valid ? fma2(cur.n.d21, sub2(cur.n.b1, kv1), vb1) : zero2;
      const T2 z22 = shfl_down2(z20);

      // ---- stage B: element row je - 1 and z3 at node row je - 1 ----
      if (je >= r0) {  // uniform over the warp
        T2 kb0, kb1;
        element_row2<S2>(a, eprev, zb0, zb1, zb2, z20, z21, bac0, bac1, bgbp0, bgbp1, bgvp0, bgvp1,
                         kb0, kb1);
        if (je > r0) {  // node row je - 1 in [r0, r1]; D^-1 is zero on clamped nodes
          const T2 z30 = fma2(nprev.d20, sub2(nprev.b0, kb0), zb0);
          const T2 z31 = fma2(nprev.d21, sub2(nprev.b1, kb1), zb1);
          st_pair(a.out, k - pitch, z30, z31, own0, own1);
        }
      } else {
        bac0 = sub2(z21, z20);  // edges of the row that becomes stage B's bottom
        bac1 = sub2(z22, z21);
      }
      zb0 = z20;
      zb1 = z21;
      zb2 = z22;
      eprev = cur.e;
      nprev = cur.n;
      vb0 = vt0;
      vb1 = vt1;
      vb2 = shfl_down2(vt0);
      k += pitch;
    }
  }
}

template <int SRC, int PF>
__device__ __forceinline__ void pre2_warp(const SweepParams<float>& a, int wg, int lane) {
  using T = float;
  using T2 = float2;
  using S2 = Sweep2<float, SRC, MODE_SMOOTH0, false, float2>;
  using VR = typename S2::VR;
  using ER = typename S2::ER;
  const int strip = wg % a.nstrips;
  const int chunk = wg / a.nstrips;
  if (chunk >= a.nchunks) return;
  const Grid g = a.g;
  const Grid gc = a.gc;
  // Lane L holds fine columns i0, i0 + 1 with i0 = 2 I, I its coarse column;
  // lanes 2-30 output coarse columns 29 strip .. 29 strip + 28.
  const int i0 = strip * (2 * PRE2_CSTRIDE) - 4 + 2 * lane;
  const int I = i0 >> 1;
  const bool col0 = i0 >= 0 && i0 <= g.nx, col1 = i0 + 1 >= 0 && i0 + 1 <= g.nx;
  const bool cfix0 = ((g.fixed & 2u) && i0 == 0) || ((g.fixed & 4u) && i0 == g.nx);
  const bool cfix1 = ((g.fixed & 2u) && i0 + 1 == 0) || ((g.fixed & 4u) && i0 + 1 == g.nx);
  const bool cout = lane >= 2 && lane <= 30 && I >= 0 && I <= gc.nx;
  // z1 goes to memory as well (the post-smoothing corrects it): lanes 2-30
  // own fine columns 58 strip .. 58 strip + 57, the task fine rows
  // 2 Jb .. 2 Je + 1.
  const bool zown0 = lane >= 2 && lane <= 30 && col0, zown1 = lane >= 2 && lane <= 30 && col1;
  // Coarse rows Jb .. Je; stage B (the residual) marches fine rows
  // jb0 .. jb1 as the restriction sweep does, stage A one row ahead.
  const int Jb = chunk * (a.H >> 1), Je = min(Jb + (a.H >> 1) - 1, gc.ny);
  const int jb0 = max(2 * Jb - 2, -1), jb1 = 2 * Je + 1;
  const int je0 = max(jb0 - 1, -1), je1 = jb1 + 1;  // stage A's steps
  const long long pitch = g.pitch;
  const T2 zero2 = make_float2(0.f, 0.f);

  struct Pack {
    VR vt;
    ER e;
  };
  auto load_pack = [&](Pack& pk, int je, long long ke) {
    S2::load_v(a, ke + pitch, i0, je + 1, pk.vt);
    S2::load_e(a, ke, i0, je, pk.e);
  };

  // Stage A (first sweep formed on the fly): z0 = w D^-1 b at the first row;
  // b and w D^-1 of node row je are carried from the previous top row.
  const long long k0 = g.at(i0, je0);
  T2 vb0, vb1, bc0, bc1, wc0, wc1;
  {
    VR r;
    S2::load_v(a, k0, i0, je0, r);
    bc0 = r.v0;
    bc1 = r.v1;
    wc0 = r.d20;
    wc1 = r.d21;
    vb0 = mul2(wc0, bc0);
    vb1 = mul2(wc1, bc1);
  }
  T2 vb2 = shfl_down2(vb0);
  T2 ac0 = sub2(vb1, vb0), ac1 = sub2(vb2, vb1);
  T2 gbp0 = zero2, gbp1 = zero2, gvp0 = zero2, gvp1 = zero2;
  // Stage B: z1 of its bottom row, edges, forces, the element data and b of
  // that row, and the partial coarse row of the restriction.
  T2 zb0 = zero2, zb1 = zero2, zb2 = zero2;
  T2 bac0 = zero2, bac1 = zero2, bgbp0 = zero2, bgbp1 = zero2, bgvp0 = zero2, bgvp1 = zero2;
  T2 bp0 = zero2, bp1 = zero2;  // b of stage B's node row
  ER eprev{};
  T2 racc = zero2;

  Pack ring[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u)
    if (je0 + u <= je1) load_pack(ring[u], je0 + u, k0 + u * pitch);

  long long k = k0;  // node (i0, je)
  for (int jb = je0; jb <= je1; jb += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int je = jb + u;
      if (je > je1) break;
      const Pack cur = ring[u];
      if (je + PF <= je1) load_pack(ring[u], je + PF, k + PF * pitch);

      // ---- stage A: z1 at node row je ----
      const T2 btop0 = cur.vt.v0, btop1 = cur.vt.v1;  // b and w D^-1 of row je + 1
      const T2 wt0 = cur.vt.d20, wt1 = cur.vt.d21;
      const T2 vt0 = mul2(wt0, btop0), vt1 = mul2(wt1, btop1);
      T2 kv0, kv1;
      element_row2<S2>(a, cur.e, vb0, vb1, vb2, vt0, vt1, ac0, ac1, gbp0, gbp1, gvp0, gvp1, kv0, kv1);
      // w D^-1, z0 and b vanish on clamped and ghost nodes, so z1 does too.
      const bool valid = je > je0;
      const T2 z10 = valid ? fma2(wc0, sub2(bc0, kv0), vb0) : zero2;
      const T2 z11 = valid ? fma2(wc1, sub2(bc1, kv1), vb1) : zero2;
      const T2 z12 = shfl_down2(z10);
      if (je >= 2 * Jb && je <= 2 * Je + 1 && je <= g.ny) st_pair(a.out, k, z10, z11, zown0, zown1);

      // ---- stage B: element row je - 1, residual at node row je - 1 ----
      const int jr = je - 1;  // stage B's row
      if (jr >= jb0) {        // uniform over the warp
        T2 kb0, kb1;
        element_row2<S2>(a, eprev, zb0, zb1, zb2, z10, z11, bac0, bac1, bgbp0, bgbp1, bgvp0, bgvp1,
                         kb0, kb1);
        if (jr > jb0) {
          const bool rowok = jr <= g.ny && !(((g.fixed & 1u) && jr == 0) || ((g.fixed & 8u) && jr == g.ny));
          const T m0 = rowok && col0 && !cfix0 ? T(1) : T(0), m1 = rowok && col1 && !cfix1 ? T(1) : T(0);
          const T2 r0 = mul2(sub2(bp0, kb0), mk2<T>(m0, m0));
          const T2 r1 = mul2(sub2(bp1, kb1), mk2<T>(m1, m1));
          // Full weighting (1/2, 1, 1/2) across, then along the march over
          // fine rows 2J - 1, 2J, 2J + 1.
          const T2 rl = shfl_up2(r1);
          const T2 h = mk2<T>(r0.x + T(0.5) * (r1.x + rl.x), r0.y + T(0.5) * (r1.y + rl.y));
          if (jr & 1) {
            const int Jlo = (jr - 1) / 2;
            const T2 val = mk2<T>(racc.x + T(0.5) * h.x, racc.y + T(0.5) * h.y);
            if (cout && Jlo >= Jb && Jlo <= Je) a.bc[gc.at(I, Jlo)] = gc.is_fixed(I, Jlo) ? zero2 : val;
            racc = mk2<T>(T(0.5) * h.x, T(0.5) * h.y);
          } else {
            racc = add2(racc, h);
          }
        }
      } else {
        bac0 = sub2(z11, z10);  // edges of the row that becomes stage B's bottom
        bac1 = sub2(z12, z11);
      }
      zb0 = z10;
      zb1 = z11;
      zb2 = z12;
      eprev = cur.e;
      bp0 = bc0;  // b of node row je: stage B's next row
      bp1 = bc1;
      bc0 = btop0;
      bc1 = btop1;
      wc0 = wt0;
      wc1 = wt1;
      vb0 = vt0;
      vb1 = vt1;
      vb2 = shfl_down2(vt0);
      k += pitch;
    }
  }
}

template <int SRC, int PF>
__global__ void __launch_bounds__(SWEEP_NT, 1) post2_kernel(const SweepParams<float> a) {
  pdl_wait();
  if (a.sc != nullptr && a.gate && a.sc->done != RUNNING) return;  // uniform over the grid
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (SWEEP_NT / 32) + (threadIdx.x >> 5);
  post2_warp<SRC, PF>(a, wg, lane);
}

template <int SRC, int PF>
__global__ void __launch_bounds__(SWEEP_NT, 1) pre2_kernel(const SweepParams<float> a) {
  pdl_wait();
  if (a.sc != nullptr && a.gate && a.sc->done != RUNNING) return;  // uniform over the grid
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (SWEEP_NT / 32) + (threadIdx.x >> 5);
  pre2_warp<SRC, PF>(a, wg, lane);
}

}  // namespace mto
