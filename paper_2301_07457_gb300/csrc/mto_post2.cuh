// Fused post-smoothing of a float32 coarse level (Alg. 1, steps after the
// coarse-grid correction): the prolongation with the first damped-Jacobi
// sweep (stage A) and the second sweep (stage B) in one marching pass.
//
// Stage A is the PSMOOTH sweep of mto_sweep2.cuh: at step je it completes
// node row je of z2 = v + w D^-1 (b - K v), v = z + P z_c.  Stage B runs one
// node row behind on the values stage A has just produced, in registers: at
// step je it evaluates element row je - 1 and completes node row je - 1 of
// z3 = z2 + w D^-1 (b - K z2), reusing the element data and the b, D^-1 that
// stage A loaded one step earlier.  z2 never goes to memory, and a level's
// post-smoothing costs one launch and one pass over its data instead of two.
//
// Each stage loses one column at each side of the warp (a value needs its
// neighbours of the stage before), so a warp outputs 60 columns (lanes 1-30)
// and stage A runs over two more rows than the chunk (rows r0 - 1 .. r1 + 1
// of z2 feed rows r0 .. r1 of z3); the halo work is recomputed by the
// neighbouring tasks.
#pragma once

#include "mto_sweep2.cuh"

namespace mto {

constexpr int POST2_STRIDE = 60;  // output columns per warp

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
  const bool cfix0 = ((g.fixed & 2u) && i0 == 0) || ((g.fixed & 4u) && i0 == g.nx);
  const bool cfix1 = ((g.fixed & 2u) && i0 + 1 == 0) || ((g.fixed & 4u) && i0 + 1 == g.nx);
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

  // One element row of a marching sweep: marched values vb (node row jj, with
  // vb2 = the right neighbour's first column) and vt (row jj + 1), bottom
  // edges ac and the edge forces gbp, gvp carried from the element row
  // below.  Returns K v at node row jj and advances the carried state.
  auto element_row = [&](const ER& e, const T2& vb0, const T2& vb1, const T2& vb2, const T2& vt0,
                         const T2& vt1, T2& ac0, T2& ac1, T2& gbp0, T2& gbp1, T2& gvp0, T2& gvp1,
                         T2& kv0, T2& kv1) {
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
  // Stage B: z2 of its bottom node row (je - 1; zero below the first row of
  // z2, which is also the value of the ghost row -1), its edges and forces,
  // and the element and node data of that row from stage A's last step.
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
      element_row(cur.e, vb0, vb1, vb2, vt0, vt1, ac0, ac1, gbp0, gbp1, gvp0, gvp1, kv0, kv1);
      // D^-1 and v vanish on clamped and ghost nodes, so z2 does too.  The
      // first step has no row below: its z2 is never used.
      const T2 z20 = fma2(cur.n.d20, sub2(cur.n.b0, kv0), vb0);
      const T2 z21 = fma2(cur.n.d21, sub2(cur.n.b1, kv1), vb1);
      const T2 z22 = shfl_down2(z20);

      // ---- stage B: element row je - 1 and z3 at node row je - 1 ----
      if (je >= r0) {  // uniform over the warp
        T2 kb0, kb1;
        element_row(eprev, zb0, zb1, zb2, z20, z21, bac0, bac1, bgbp0, bgbp1, bgvp0, bgvp1, kb0, kb1);
        if (je > r0) {
          const int jo = je - 1;  // r0 <= jo <= r1
          const bool rfix = ((g.fixed & 1u) && jo == 0) || ((g.fixed & 8u) && jo == g.ny);
          (void)rfix;  // D^-1 is zero on clamped nodes: z3 = z2 = 0 there
          const T2 z30 = fma2(nprev.d20, sub2(nprev.b0, kb0), zb0);
          const T2 z31 = fma2(nprev.d21, sub2(nprev.b1, kb1), zb1);
          st_pair(a.out, k - pitch, z30, z31, own0, own1);
        }
      } else {
        bac0 = sub2(z21, z20);  // edges of the row that becomes stage B's bottom
        bac1 = sub2(z22, z21);
      }
      (void)cfix0;
      (void)cfix1;
      zb0 = je > je0 ? z20 : zero2;
      zb1 = je > je0 ? z21 : zero2;
      zb2 = je > je0 ? z22 : zero2;
      if (!(je > je0)) {
        bac0 = zero2;
        bac1 = zero2;
      }
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
__global__ void __launch_bounds__(SWEEP_NT, 1) post2_kernel(const SweepParams<float> a) {
  pdl_wait();
  if (a.sc != nullptr && a.gate && a.sc->done != RUNNING) return;  // uniform over the grid
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (SWEEP_NT / 32) + (threadIdx.x >> 5);
  post2_warp<SRC, PF>(a, wg, lane);
}

}  // namespace mto
