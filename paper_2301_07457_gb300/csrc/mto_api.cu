// C ABI of libmto: context and memory plan, per-design setup, the PCG driver
// (Alg. 2) with its V-cycle preconditioner (Alg. 1), compliance and
// sensitivities, and the diagnostic entry points.
//
// A solve is one CUDA graph: the PCG loop runs on the device inside a
// conditional WHILE node whose body holds two iterations; the last kernel of
// the body keeps the loop going while the device scalars say "running".  No
// host round trip happens inside a solve.  With kernel timing on, the loop is
// driven from the host instead (graph of two iterations, polled), because
// event records cannot live inside a conditional body.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "mto_ctx.cuh"

using namespace mto;

thread_local cudaError_t mto::g_last_cuda = cudaSuccess;

namespace {
std::mutex g_mem_mutex;
std::map<void*, size_t> g_mem_blocks;
size_t g_mem_in_use = 0, g_mem_limit = 0;
}  // namespace

namespace mto {

cudaError_t device_alloc(void** p, size_t bytes) {
  *p = nullptr;
  std::lock_guard<std::mutex> lock(g_mem_mutex);
  if (g_mem_limit && g_mem_in_use + bytes > g_mem_limit) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  g_mem_blocks[*p] = bytes;
  g_mem_in_use += bytes;
  return cudaSuccess;
}

void device_free(void* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(g_mem_mutex);
    auto it = g_mem_blocks.find(p);
    if (it != g_mem_blocks.end()) {
      g_mem_in_use -= it->second;
      g_mem_blocks.erase(it);
    }
  }
  cudaFree(p);
}

}  // namespace mto

namespace {

mto_status dalloc(mto_ctx* c, void** out, size_t bytes) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  if (device_alloc(out, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MTO_ERR_OOM;
  }
  c->allocs.push_back(*out);
  // The zero fill runs on the legacy stream, which the context's non-blocking
  // streams do not order against: wait for it here.
  if (cudaMemset(*out, 0, bytes) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess)
    return MTO_ERR_CUDA;
  return MTO_OK;
}

template <typename P> mto_status dalloc_t(mto_ctx* c, P** out, size_t count) {
  void* v = nullptr;
  mto_status s = dalloc(c, &v, count * sizeof(P));
  *out = static_cast<P*>(v);
  return s;
}

// Make the context's stream wait for the caller's stream, and back.
mto_status enter(mto_ctx* c) {
  CK(cudaSetDevice(c->device));
  CK(cudaEventRecord(c->ev_in, c->user_stream));
  CK(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  c->cs = c->stream;
  return MTO_OK;
}
mto_status leave(mto_ctx* c) {
  CK(cudaEventRecord(c->ev_out, c->stream));
  CK(cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
  return MTO_OK;
}

}  // namespace

namespace mto {

int target_warps(const mto_ctx* c, int level) {
  return (level >= 0 && level < MAX_LEVELS) ? c->tw[level] : 0;
}

int target_warps64(const mto_ctx* c) { return c->tw64; }

void invalidate_graphs(mto_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
  c->gexec = nullptr;
  c->solve_exec = nullptr;
  for (mto_ctx* s : c->slots) invalidate_graphs(s);
}

}  // namespace mto

namespace {

// ---------------------------------------------------------------------------
// Sweep helpers
// ---------------------------------------------------------------------------
template <typename T> SweepParams<T> base_params(const mto_ctx* c, const Grid& g) {
  SweepParams<T> p;
  std::memset(&p, 0, sizeof(p));
  p.g = g;
  p.cstride = g.size();
  p.partials = c->partials;
  p.ticket = c->ticket;
  return p;
}

template <typename T> FineConst<T> fine_const(const mto_ctx* c);
template <> FineConst<double> fine_const<double>(const mto_ctx* c) { return c->kf64; }
template <> FineConst<float> fine_const<float>(const mto_ctx* c) { return c->kf32; }

// SRC_CMOM parameters: nu and g = (1 - nu) / 2.
template <typename T> void set_cmom(const mto_ctx* c, SweepParams<T>& p) {
  p.cnu = T(c->nu);
  p.cg = T(0.5 * (1.0 - c->nu));
}

// SRC_CFINE parameters: the finest bf16 moduli and their grid.
template <typename T> void set_cfine(const mto_ctx* c, SweepParams<T>& p) {
  p.E = c->Ebf;
  p.gfine = c->lv[c->L].g;
  p.kf = fine_const<T>(c);
  p.redisc = c->o.coarse_kind == MTO_COARSE_REDISCRETIZE;
}

template <typename T> mto_status coarse_calls(mto_ctx* c, int l, int calls, DevScalars* sc,
                                               int* final_idx);

// One call MG^l(U_l, F_l) of Alg. 1 on coarse level l >= 1 with right-hand
// side lv[l].b: from U_l = 0 when start < 0, else from the iterate in
// lv[l].z[start] (the repeated calls of a W-cycle).  Returns the index of the
// z buffer that holds the result.
template <typename T>
mto_status coarse_cycle(mto_ctx* c, int l, DevScalars* sc, int start, int* final_idx) {
  using T2 = typename V2<T>::t;
  LevelBuf& L = c->lv[l];
  LevelBuf& C = c->lv[l - 1];
  const int tw = target_warps(c, l);
  const int nb = vec_blocks(L.g.size(), c->num_sms);
  int cur = 0;
  // The first coarse level of the mixed path rebuilds its element matrices
  // from the bf16 fine moduli (SRC_CFINE); other coarse levels read stored
  // coefficients.
  const bool cfine = sizeof(T) == 4 && l == c->L - 1;
  const int src = cfine ? SRC_CFINE : (sizeof(T) == 4 ? SRC_CMOM : SRC_COARSE);
  auto sweep = [&](int mode, const T2* v, T2* out, const T2* zc) -> cudaError_t {
    SweepParams<T> p = base_params<T>(c, L.g);
    p.gc = C.g;
    p.gate = 1;
    p.sc = sc;
    p.v = v;
    p.zc = zc;
    p.b = (const T2*)L.b;
    p.out = out;
    p.bc = (T2*)C.b;
    p.coef = (const T*)L.coef;
    p.invd2 = (const T2*)L.invd2;
    set_cmom(c, p);
    if (cfine) set_cfine(c, p);
    return launch_sweep<T>(src, mode, false, false, p, tw, c->num_sms, c->cs);
  };
  // Pre-smoothing from U = 0: the first sweep (U = w D^-1 F) is formed on the
  // fly inside the second when there are two or more.  With exactly two on a
  // float32 level, the residual and its restriction run in the same pass
  // (mto_fused.cuh).
  const bool fused_pre = (src == SRC_CMOM || src == SRC_CFINE) && c->o.nu1 == 2;
  if (start >= 0) {
    cur = start;
    for (int s = 0; s < c->o.nu1; ++s) {
      KL(sweep(MODE_SMOOTH, (const T2*)L.z[cur], (T2*)L.z[cur ^ 1], nullptr));
      cur ^= 1;
    }
    KL(sweep(MODE_RESTRICT, (const T2*)L.z[cur], nullptr, nullptr));
  } else if (fused_pre) {
    KL(sweep(MODE_PRE2, nullptr, (T2*)L.z[0], nullptr));
  } else {
    if (c->o.nu1 >= 2) {
      KL(sweep(MODE_SMOOTH0, nullptr, (T2*)L.z[0], nullptr));
    } else {
      KL(launch_jacobi0_coarse<T>(L.g, (const T2*)L.invd2, (const T2*)L.b, (T2*)L.z[0], sc, nb,
                                  c->cs));
    }
    for (int s = 2; s < c->o.nu1; ++s) {
      KL(sweep(MODE_SMOOTH, (const T2*)L.z[cur], (T2*)L.z[cur ^ 1], nullptr));
      cur ^= 1;
    }
    KL(sweep(MODE_RESTRICT, (const T2*)L.z[cur], nullptr, nullptr));
  }
  int cidx = 0;
  ST(coarse_calls<T>(c, l - 1, c->o.gamma, sc, &cidx));
  // Post-smoothing; on the float32 levels the prolongation sweep and the
  // next one run fused (mto_fused.cuh).
  int s = 1;
  if ((src == SRC_CMOM || src == SRC_CFINE) && c->o.nu2 >= 2) {
    KL(sweep(MODE_POST2, (const T2*)L.z[cur], (T2*)L.z[cur ^ 1], (const T2*)C.z[cidx]));
    s = 2;
  } else {
    KL(sweep(MODE_PSMOOTH, (const T2*)L.z[cur], (T2*)L.z[cur ^ 1], (const T2*)C.z[cidx]));
  }
  cur ^= 1;
  for (; s < c->o.nu2; ++s) {
    KL(sweep(MODE_SMOOTH, (const T2*)L.z[cur], (T2*)L.z[cur ^ 1], nullptr));
    cur ^= 1;
  }
  *final_idx = cur;
  return MTO_OK;
}

// "Call the scheme gamma times for the next coarser grid" (Alg. 1) on level
// l, each call continuing from the iterate the previous one returned.  On
// the coarsest grid the scheme is the exact solve U_0 = K_0^-1 F_0, which
// does not depend on the iterate: one GEMV stands for all calls.
template <typename T>
mto_status coarse_calls(mto_ctx* c, int l, int calls, DevScalars* sc, int* final_idx) {
  using T2 = typename V2<T>::t;
  if (l == 0) {
    LevelBuf& C = c->lv[0];
    KL(launch_coarsest_gemv<T>(C.g, c->n0, c->dof_index + 2 * C.g.size(), c->Kinv, (const T2*)C.b,
                               (T2*)C.z[0], sc, c->cs));
    *final_idx = 0;
    return MTO_OK;
  }
  int idx = -1;
  for (int k = 0; k < calls; ++k) ST(coarse_cycle<T>(c, l, sc, idx, &idx));
  *final_idx = idx;
  return MTO_OK;
}

// Whether the mixed-precision PCG step leaves r -= alpha q to the next
// V-cycle's first smoothing sweep (FIN_PQ_FUSED / FIN_UPDATE_FUSED): that
// sweep loads r anyway (as its float32 copy), and the update's FP64 work
// overlaps the sweep's float32 work.
bool fuse_update(const mto_ctx* c) { return c->mixed && c->o.nu1 >= 2; }

// Residual of the PCG step of parity par (the buffers alternate only when
// the update is fused).
double2* rbuf(const mto_ctx* c, int par) { return (fuse_update(c) && par == 1) ? c->r_alt : c->r; }

// V-cycle on the finest level with right-hand side r (float64).  With
// with_dot (inside the PCG loop), the last post-smoothing sweep also forms
// z.r (and z.q) and finishes beta (FIN_RHO), and with fuse_update the first
// sweep applies the pending CG update of r.
template <typename T>
mto_status fine_cycle(mto_ctx* c, DevScalars* sc, bool with_dot, int* final_idx) {
  using T2 = typename V2<T>::t;
  constexpr bool MIX = sizeof(T) == 4;
  LevelBuf& L = c->lv[c->L];
  LevelBuf& C = c->lv[c->L - 1];
  const int tw = target_warps(c, c->L);
  const int nb = vec_blocks(L.g.size(), c->num_sms);
  const int src = MIX ? SRC_FINEBF : SRC_FINE64;
  // The first pre-sweep from zero is fused into the second (SMOOTH0) when
  // there are two or more.  The mixed cycle reads the float32 copy of r that
  // the kernels writing r (CG update, residuals) keep next to it.
  const T2* b = MIX ? (const T2*)c->r32 : (const T2*)c->r;
  const bool fused0 = c->o.nu1 >= 2;
  if (!fused0) {
    if constexpr (MIX) {
      KL(launch_jacobi0_finebf(L.g, c->Ebf, (float)c->w_over_kdiag, c->r32, (float2*)L.z[0], sc, nb,
                               c->cs));
    } else {
      KL(launch_jacobi0_fine64(L.g, c->invd1, c->r, (double2*)L.z[0], sc, nb, c->cs));
    }
  }
  int cur = 0;
  auto sweep = [&](int mode, const T2* v, T2* out, const T2* zc, bool dot) -> cudaError_t {
    SweepParams<T> p = base_params<T>(c, L.g);
    p.gc = C.g;
    p.gate = 1;
    p.sc = sc;
    p.v = v;
    p.zc = zc;
    p.b = b;
    p.out = out;
    p.bc = (T2*)C.b;
    p.E = MIX ? (const void*)c->Ebf : (const void*)c->Ek4;
    p.kf = fine_const<T>(c);
    p.invd1 = c->invd1;
    p.wdiag = T(c->w_over_kdiag);
    if (dot && mode == MODE_SMOOTH0) {
      // The CG update r -= alpha q of the last step (mixed precision).
      p.r64 = rbuf(c, c->cur_par);
      p.r64_prev = rbuf(c, c->cur_par ^ 1);
      p.q64 = c->q;
      p.out32 = c->r32;
      p.finish = FIN_UPDATE_FUSED;
    } else if (dot) {
      p.rdot = rbuf(c, c->cur_par);
      p.qdot = c->o.flexible ? c->q : nullptr;
      p.finish = FIN_RHO;
    }
    return launch_sweep<T>(src, mode, dot, false, p, tw, c->num_sms, c->cs);
  };
  // Timing events bracket the first finest-level smoothing kernel.
  const bool tm = c->timing && sc != nullptr && c->cur_par >= 0;
  auto t0 = [&]() -> cudaError_t {
    return tm ? cudaEventRecordWithFlags(c->kev[c->cur_par][1][0], c->cs, cudaEventRecordExternal)
              : cudaSuccess;
  };
  auto t1 = [&]() -> cudaError_t {
    return tm ? cudaEventRecordWithFlags(c->kev[c->cur_par][1][1], c->cs, cudaEventRecordExternal)
              : cudaSuccess;
  };
  int first = 1;
  if (fused0) {
    CK(t0());
    KL(sweep(MODE_SMOOTH0, nullptr, (T2*)L.z[0], nullptr, fuse_update(c) && with_dot));
    CK(t1());
    first = 2;
  }
  for (int s = first; s < c->o.nu1; ++s) {
    if (s == 1) CK(t0());
    KL(sweep(MODE_SMOOTH, (const T2*)L.z[cur], (T2*)L.z[cur ^ 1], nullptr, false));
    if (s == 1) CK(t1());
    cur ^= 1;
  }
  KL(sweep(MODE_RESTRICT, (const T2*)L.z[cur], nullptr, nullptr, false));
  // Alg. 1 calls the next coarser grid once from the finest grid.
  int cidx = 0;
  ST(coarse_calls<T>(c, c->L - 1, 1, sc, &cidx));
  KL(sweep(MODE_PSMOOTH, (const T2*)L.z[cur], (T2*)L.z[cur ^ 1], (const T2*)C.z[cidx],
           with_dot && c->o.nu2 == 1));
  cur ^= 1;
  for (int s = 1; s < c->o.nu2; ++s) {
    KL(sweep(MODE_SMOOTH, (const T2*)L.z[cur], (T2*)L.z[cur ^ 1], nullptr,
             with_dot && s == c->o.nu2 - 1));
    cur ^= 1;
  }
  *final_idx = cur;
  return MTO_OK;
}

// out = b - K v on the finest level in float64 (RESID), with a finishing action.
// With xlag, the sweep works on v + alpha xdir while the device scalars say
// that the x step is pending (residual replacement inside the loop).
mto_status fine_resid(mto_ctx* c, const double2* v, const double2* b, double2* out, int finish,
                      int gate, int replace_gate, int zero_gate = 0, int xlag = 0,
                      const double2* xdir = nullptr) {
  const Grid& g = c->lv[c->L].g;
  SweepParams<double> p = base_params<double>(c, g);
  p.gate = gate;
  p.replace_gate = replace_gate;
  p.zero_gate = zero_gate;
  p.sc = c->sc;
  p.v = v;
  p.b = b;
  p.out = out;
  p.E = c->Ek4;
  p.finish = finish;
  p.xlag = xlag;
  p.xdir = xdir;
  if (c->mixed && (out == c->r || out == c->r_alt)) p.out32 = c->r32;
  KL(launch_sweep<double>(SRC_FINE64, MODE_RESID, false, false, p,
                          target_warps64(c), c->num_sms, c->cs));
  return MTO_OK;
}

// One PCG iteration (Alg. 2) with search directions p[par] -> p[par ^ 1].
mto_status enqueue_iteration(mto_ctx* c, int par) {
  const Grid& g = c->lv[c->L].g;
  c->cur_par = par;
  int zi = 0;
  if (c->mixed) {
    ST(fine_cycle<float>(c, c->sc, true, &zi));
  } else {
    ST(fine_cycle<double>(c, c->sc, true, &zi));
  }
  const void* z = c->lv[c->L].z[zi];
  // External event-record nodes inside the captured graph (a plain record
  // during capture would only mark a dependency).
  if (c->timing) CK(cudaEventRecordWithFlags(c->kev[par][0][0], c->cs, cudaEventRecordExternal));
  {
    SweepParams<double> p = base_params<double>(c, g);
    p.gate = 1;
    p.sc = c->sc;
    p.v = c->p[par];
    p.zkp = z;
    p.p_out = c->p[par ^ 1];
    p.xvec = c->x;
    p.tag = par ^ 1;
    p.out = c->q;
    p.E = c->Ek4;
    p.finish = fuse_update(c) ? FIN_PQ_FUSED : FIN_PQ;
    KL(launch_sweep<double>(SRC_FINE64, MODE_KP, false, c->mixed, p,
                            target_warps64(c), c->num_sms, c->cs));
  }
  if (c->timing) CK(cudaEventRecordWithFlags(c->kev[par][0][1], c->cs, cudaEventRecordExternal));
  if (!fuse_update(c))
    KL(launch_update(g, c->r, c->mixed ? c->r32 : nullptr, c->q, c->partials, c->ticket, c->sc,
                     vec_blocks(g.size(), c->num_sms), c->cs));
  if (c->mixed && c->o.rr_every > 0)
    ST(fine_resid(c, c->x, c->f, rbuf(c, par ^ 1), FIN_REPLACE, 1, 1, 0, 1, c->p[par ^ 1]));
  return MTO_OK;
}

// Graph of two iterations for the host-polled loop.
mto_status build_poll_graph(mto_ctx* c) {
  if (c->gexec) return MTO_OK;
  cudaGraph_t graph = nullptr;
  c->cs = c->stream;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  const long long before = c->launches;
  mto_status s0 = enqueue_iteration(c, 0);
  mto_status s1 = s0 == MTO_OK ? enqueue_iteration(c, 1) : s0;
  c->cur_par = -1;
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  c->graph_kernels = c->launches - before;
  c->launches = before;
  if (s1 != MTO_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return s1;
  }
  if (e != cudaSuccess) {
    g_last_cuda = e;
    return MTO_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&c->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->gexec = nullptr;
    g_last_cuda = e;
    return MTO_ERR_CUDA;
  }
  return MTO_OK;
}

// Graph of a whole solve (everything after the packing of f and u).
mto_status build_solve_graph(mto_ctx* c) {
  if (c->solve_exec) return MTO_OK;
  cudaGraph_t graph = nullptr;
  c->cs = c->stream;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  const long long before = c->launches;
  mto_status s = enqueue_solve_core(c);
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  c->solve_kernels_fixed = c->launches - before;
  c->launches = before;
  c->cs = c->stream;
  if (s != MTO_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (s == MTO_OK) g_last_cuda = e;
    return s != MTO_OK ? s : MTO_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&c->solve_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->solve_exec = nullptr;
    g_last_cuda = e;
    return MTO_ERR_CUDA;
  }
  return MTO_OK;
}

// Host-polled solve loop (kernel timing mode, or no conditional nodes).
mto_status solve_polled(mto_ctx* c) {
  const Grid& g = c->lv[c->L].g;
  CK(cudaMemsetAsync(c->p[0], 0, sizeof(double2) * g.size(), c->stream));
  KL(launch_dot(g.size(), c->f, c->f, c->partials, c->ticket, c->sc, FIN_FF, nullptr,
                vec_blocks(g.size(), c->num_sms), c->stream));
  ST(fine_resid(c, c->x, c->f, c->r, FIN_INIT_RR, 0, 0, 1));
  ST(build_poll_graph(c));
  const int poll = (c->o.check_every + 1) / 2;  // graph launches (2 iterations each) per poll
  int launched = 0;
  for (;;) {
    CK(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->timing && launched > 0 && c->sc_host->done == RUNNING) {
      // Every iteration of the last graph launch ran in full: sample it.
      for (int par = 0; par < 2; ++par)
        for (int k = 0; k < 2; ++k) {
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, c->kev[par][k][0], c->kev[par][k][1]) == cudaSuccess) {
            c->ksum[k] += ms;
            c->kcnt[k] += 1;
          } else {
            cudaGetLastError();  // a missing sample is not a failure of the solve
          }
        }
    }
    if (c->sc_host->done != RUNNING || launched > c->o.max_it + 2) break;
    for (int k = 0; k < poll; ++k) {
      CK(cudaGraphLaunch(c->gexec, c->stream));
      c->launches += c->graph_kernels;
      launched += 2;
    }
  }
  KL(launch_x_step(g, c->x, c->p[0], c->p[1], c->sc, vec_blocks(g.size(), c->num_sms), c->stream));
  ST(fine_resid(c, c->x, c->f, c->tmp, FIN_TRUE, 0, 0));
  return MTO_OK;
}

// Coarse-level calls of one cycle below the finest level (the coarsest grid
// excluded): once on the next grid, gamma times on the one below, and so on.
// Each call adds a few kernels to the solve graph, so the count is capped.
constexpr long MAX_COARSE_VISITS = 512;
long coarse_visits(int n_coarsen, int gamma) {
  long visits = 0, per = 1;
  for (int l = n_coarsen - 1; l >= 1 && visits <= MAX_COARSE_VISITS; --l, per *= gamma)
    visits += per;
  return visits;
}

bool valid_opts(const mto_solver_opts& o) {
  return o.tol >= 0.0 && o.max_it >= 0 && o.omega > 0.0 && o.omega <= 1.0 && o.nu1 >= 1 &&
         o.nu2 >= 1 && o.nu1 <= 16 && o.nu2 <= 16 && o.n_coarsen >= 1 && o.n_coarsen <= 14 &&
         (o.coarse_kind == MTO_COARSE_GALERKIN || o.coarse_kind == MTO_COARSE_REDISCRETIZE) &&
         (o.precision == MTO_PRECISION_FP64 || o.precision == MTO_PRECISION_MIXED) &&
         o.rr_every >= 0 && o.check_every >= 1 && o.gamma >= 1 && o.gamma <= 4 &&
         o.concurrent_rhs >= 1 && o.concurrent_rhs <= MAX_CONCURRENT_RHS &&
         coarse_visits(o.n_coarsen, o.gamma) <= MAX_COARSE_VISITS;
}

mto_status status_of(const RhsStats& r) {
  if (r.done == BREAKDOWN) return MTO_ERR_BREAKDOWN;
  if (r.done != CONVERGED) return MTO_ERR_NOT_CONVERGED;
  return MTO_OK;
}

}  // namespace

// ===========================================================================
// Enqueue functions shared with the batch driver (capturable: no host sync).
// ===========================================================================
namespace mto {

mto_status enqueue_solve_core(mto_ctx* c) {
  const Grid& g = c->lv[c->L].g;
  CK(cudaMemsetAsync(c->p[0], 0, sizeof(double2) * g.size(), c->cs));
  KL(launch_dot(g.size(), c->f, c->f, c->partials, c->ticket, c->sc, FIN_FF, nullptr,
                vec_blocks(g.size(), c->num_sms), c->cs));
  ST(fine_resid(c, c->x, c->f, c->r, FIN_INIT_RR, 0, 0, 1));
  // Device-side loop: a conditional WHILE node after the current capture
  // dependencies, its body captured on the body stream.
  cudaStreamCaptureStatus st;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(c->cs, &st, nullptr, &graph, &deps, &edges, &nd));
  if (st != cudaStreamCaptureStatusActive) return MTO_ERR_STATE;
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, graph, deps, edges, nd, &np));
  CK(cudaStreamUpdateCaptureDependencies(c->cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t outer = c->cs;
  CK(cudaStreamBeginCaptureToGraph(c->body_stream, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  c->cs = c->body_stream;
  const long long before = c->launches;
  mto_status s = enqueue_iteration(c, 0);
  if (s == MTO_OK) s = enqueue_iteration(c, 1);
  if (s == MTO_OK) {
    c->launches += 1;
    const cudaError_t e = launch_set_continue(h, c->sc, c->cs);
    if (e != cudaSuccess) {
      g_last_cuda = e;
      s = MTO_ERR_CUDA;
    }
  }
  c->cur_par = -1;
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->body_stream, &captured);
  c->cs = outer;
  c->body_kernels = c->launches - before;
  c->launches = before;
  if (s != MTO_OK) return s;
  if (e != cudaSuccess) {
    g_last_cuda = e;
    return MTO_ERR_CUDA;
  }
  KL(launch_x_step(g, c->x, c->p[0], c->p[1], c->sc, vec_blocks(g.size(), c->num_sms), c->cs));
  ST(fine_resid(c, c->x, c->f, c->tmp, FIN_TRUE, 0, 0));
  return MTO_OK;
}

mto_status enqueue_rhs_prologue(mto_ctx* c, const double* f_dev, const double* u_dev) {
  const Grid& g = c->lv[c->L].g;
  KL(launch_init_scalars(c->sc, c->o.tol * c->o.tol, c->o.max_it, c->o.flexible,
                         c->mixed ? c->o.rr_every : 0, c->cs));
  KL(launch_pack(g, f_dev, c->f, c->cs, c->num_sms));
  KL(launch_pack(g, u_dev, c->x, c->cs, c->num_sms, &c->sc->x_nonzero));
  return MTO_OK;
}

mto_status enqueue_rhs_epilogue(mto_ctx* c, double* u_dev, int rhs_slot) {
  const Grid& g = c->lv[c->L].g;
  KL(launch_unpack(g, c->x, u_dev, c->cs, c->num_sms));
  KL(launch_record_stats(c->sc, c->rhs_stats + rhs_slot, c->cs));
  return MTO_OK;
}

// Design parameters of the next set_design (host side only).
void design_params(mto_ctx* c, int n_phase, const double* E_phase, double penal) {
  c->n_phase = n_phase;
  for (int i = 0; i < 16; ++i) c->ph.E[i] = i < n_phase ? E_phase[i] : 0.0;
  c->penal = penal;
  c->ipenal = (penal == std::floor(penal) && penal <= 16.0) ? (int)penal : -1;
}

// Finest moduli of element rows [j0, j1) from the design copy c->xdes.
mto_status enqueue_modulus(mto_ctx* c, int j0, int j1) {
  const Grid& gf = c->lv[c->L].g;
  KL(launch_modulus(gf, c->n_phase, c->xdes, c->ph, c->penal, c->ipenal, c->E64, c->Ebf, c->Ek4,
                    c->kf64, c->cs, c->num_sms, j0, j1));
  return MTO_OK;
}

// Everything of set_design after the finest moduli: the coarse hierarchy,
// the smoothers' diagonals and the coarsest factor and inverse.
mto_status enqueue_hierarchy(mto_ctx* c);

mto_status enqueue_set_design(mto_ctx* c, int n_phase, const double* x_dev, const double* E_phase,
                              double penal) {
  const size_t nel = (size_t)c->nelx * c->nely;
  if (c->xdes_cap < (size_t)n_phase * nel) return MTO_ERR_STATE;  // grown by the caller
  design_params(c, n_phase, E_phase, penal);
  CK(cudaMemcpyAsync(c->xdes, x_dev, sizeof(double) * n_phase * nel, cudaMemcpyDeviceToDevice, c->cs));
  ST(enqueue_modulus(c, 0, c->nely));
  return enqueue_hierarchy(c);
}

mto_status enqueue_hierarchy(mto_ctx* c) {
  const Grid& gf = c->lv[c->L].g;
  const int redisc = c->o.coarse_kind == MTO_COARSE_REDISCRETIZE;
  // Moments down the hierarchy (each level from the one above).
  for (int l = c->L - 1; l >= 0; --l) {
    LevelBuf& B = c->lv[l];
    if (l == c->L - 1) {
      KL(launch_moments_from_fine(B.g, gf, c->mixed ? nullptr : c->E64, c->mixed ? c->Ebf : nullptr,
                                  redisc, B.mom, c->cs, c->num_sms));
    } else {
      KL(launch_moments_from_coarse(B.g, c->lv[l + 1].g, c->lv[l + 1].mom, redisc, B.mom, c->cs,
                                    c->num_sms));
    }
  }
  // The coarsest factor and inverse (one SM for the factor, a serial chain)
  // run on a side stream while this one prepares the smoothers and the
  // element data of the other levels, which they do not depend on.
  LevelBuf& B0 = c->lv[0];
  KL(launch_coefs<double>(B0.g, B0.mom, c->nu, B0.coef64, c->cs, c->num_sms));
  CK(cudaMemsetAsync(c->Kd, 0, sizeof(double) * c->n0 * (c->bw0 + 1), c->cs));
  CK(cudaMemsetAsync(c->err_flag, 0, sizeof(int), c->cs));
  KL(launch_band_assemble(B0.g, B0.coef64, c->dof_index, c->n0, c->bw0, c->Kd, c->cs));
  CK(cudaEventRecord(c->ev_fork, c->cs));
  CK(cudaStreamWaitEvent(c->fac_stream, c->ev_fork, 0));
  KL(launch_cholesky_inverse(c->n0, c->bw0, c->Kd, c->invL, c->Lsc, c->Kinv, c->err_flag, c->fac_stream,
                             c->num_sms));
  c->launches += 1;  // the inverse is a second kernel
  CK(cudaEventRecord(c->ev_join, c->fac_stream));
  if (!c->mixed) KL(launch_fine_invd(gf, c->E64, c->w_over_kdiag, c->invd1, c->cs, c->num_sms));
  for (int l = c->L - 1; l >= 1; --l) {
    LevelBuf& B = c->lv[l];
    if (c->mixed) {
      // Level L-1 rebuilds its elements from the bf16 fine moduli; deeper
      // levels read scaled moments; level 0 is solved directly.
      if (l < c->L - 1) KL(launch_kmom(B.g, B.mom, c->nu, (float*)B.coef, c->cs, c->num_sms));
      KL(launch_coarse_invd<float>(B.g, B.mom, c->nu, c->o.omega, (float2*)B.invd2, c->cs, c->num_sms));
    } else {
      KL(launch_coefs<double>(B.g, B.mom, c->nu, (double*)B.coef, c->cs, c->num_sms));
      KL(launch_coarse_invd<double>(B.g, B.mom, c->nu, c->o.omega, (double2*)B.invd2, c->cs,
                                    c->num_sms));
    }
  }
  if (!c->mixed)  // the float64 level-0 coefficients of the sweeps (apply_operator)
    KL(launch_coefs<double>(B0.g, B0.mom, c->nu, (double*)B0.coef, c->cs, c->num_sms));
  CK(cudaStreamWaitEvent(c->cs, c->ev_join, 0));
  return MTO_OK;
}

mto_status enqueue_compliance(mto_ctx* c, int n_rhs, const double* f_dev, const double* u_dev,
                              double* compliance_dev, double* dcdx_dev) {
  const long long nn = (long long)(c->nelx + 1) * (c->nely + 1);
  for (int k = 0; k < n_rhs; ++k) {
    const double2* fk = reinterpret_cast<const double2*>(f_dev + 2 * nn * k);
    const double2* uk = reinterpret_cast<const double2*>(u_dev + 2 * nn * k);
    KL(launch_dot(nn, fk, uk, c->partials, c->ticket, nullptr, FIN_NONE, compliance_dev + k,
                  vec_blocks(nn, c->num_sms), c->cs));
    if (dcdx_dev)
      KL(launch_sensitivity(c->nelx, c->nely, c->n_phase, c->xdes, c->ph, c->penal, c->ipenal,
                            c->kf64, u_dev + 2 * nn * k, dcdx_dev, k > 0, c->cs, c->num_sms));
  }
  return MTO_OK;
}

}  // namespace mto

namespace {

mto_status grow(mto_ctx* c, double** p, size_t* cap, size_t need) {
  if (*cap >= need) return MTO_OK;
  ST(dalloc_t(c, p, need));
  *cap = need;
  return MTO_OK;
}

mto_status set_design_sync(mto_ctx* c, int n_phase, const double* x_dev, const double* E_phase,
                           double penal) {
  const size_t nel = (size_t)c->nelx * c->nely;
  ST(grow(c, &c->xdes, &c->xdes_cap, (size_t)n_phase * nel));
  c->cs = c->stream;
  CK(cudaEventRecord(c->ev_a, c->stream));
  ST(enqueue_set_design(c, n_phase, x_dev, E_phase, penal));
  CK(cudaMemcpyAsync(c->err_host, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaEventRecord(c->ev_b, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaEventElapsedTime(&c->ms_setup, c->ev_a, c->ev_b));
  if (*c->err_host) return MTO_ERR_BREAKDOWN;
  c->has_design = true;
  return MTO_OK;
}

// Reduction scratch: two partials per block of the largest launch.
size_t partials_count(const mto_ctx* c) {
  const Grid& gf = c->lv[c->L].g;
  int maxb = vec_blocks(gf.size(), c->num_sms);
  for (int mode = 0; mode <= MODE_RESTRICT; ++mode) {
    for (int cols = 1; cols <= 2; ++cols) {
      const SweepShape s = sweep_shape(gf, mode, MAX_TARGET_WARPS_PER_SM * c->num_sms, cols);
      if (s.nblocks > maxb) maxb = s.nblocks;
    }
  }
  return 2 * (size_t)maxb + 2;
}

// A workspace for one more concurrent right-hand side: the design data of c
// is shared (read only during a solve), the solve's vectors, scalars,
// streams and graphs are its own.  Its rhs_stats point into c's, so that
// every right-hand side records its statistics in c's array.
mto_status make_slot(mto_ctx* c, mto_ctx** out) {
  *out = nullptr;
  mto_ctx* s = new (std::nothrow) mto_ctx();
  if (!s) return MTO_ERR_OOM;
  auto fail = [&](mto_status st) {
    cudaGetLastError();
    mto_destroy(s);
    return st;
  };
  s->parent = c;
  s->device = c->device;
  s->num_sms = c->num_sms;
  s->nelx = c->nelx;
  s->nely = c->nely;
  s->nu = c->nu;
  s->fixed = c->fixed;
  s->o = c->o;
  s->L = c->L;
  s->mixed = c->mixed;
  s->kf64 = c->kf64;
  s->kf32 = c->kf32;
  s->w_over_kdiag = c->w_over_kdiag;
  s->n0 = c->n0;
  s->bw0 = c->bw0;
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->body_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_slot, cudaEventDisableTiming) != cudaSuccess)
    return fail(MTO_ERR_CUDA);
  s->cs = s->stream;
  // Shared design data.
  s->lv.resize(c->L + 1);
  for (int l = 0; l <= c->L; ++l) {
    s->lv[l].g = c->lv[l].g;
    s->lv[l].coef = c->lv[l].coef;
    s->lv[l].invd2 = c->lv[l].invd2;
    s->lv[l].mom = c->lv[l].mom;
    s->lv[l].coef64 = c->lv[l].coef64;
  }
  s->E64 = c->E64;
  s->Ek4 = c->Ek4;
  s->Ebf = c->Ebf;
  s->invd1 = c->invd1;
  s->dof_index = c->dof_index;
  s->Kd = c->Kd;
  s->Kinv = c->Kinv;
  s->invL = c->invL;
  s->Lsc = c->Lsc;
  s->err_flag = c->err_flag;
  s->rhs_stats = c->rhs_stats;
  // Own solve data.
  const size_t vsz = c->mixed ? sizeof(float2) : sizeof(double2);
  mto_status st = MTO_OK;
  for (int l = 0; l <= c->L && st == MTO_OK; ++l) {
    const size_t n = (size_t)s->lv[l].g.size();
    st = dalloc(s, &s->lv[l].z[0], n * vsz);
    if (st == MTO_OK) st = dalloc(s, &s->lv[l].z[1], n * vsz);
    if (st == MTO_OK && l < c->L) st = dalloc(s, &s->lv[l].b, n * vsz);
  }
  const size_t nf = (size_t)s->lv[c->L].g.size();
  if (st == MTO_OK && c->mixed) st = dalloc_t(s, &s->r32, nf);
  if (st == MTO_OK && c->mixed) st = dalloc_t(s, &s->r_alt, nf);
  double2** vecs[] = {&s->x, &s->r, &s->q, &s->f, &s->tmp, &s->p[0], &s->p[1]};
  for (double2** v : vecs)
    if (st == MTO_OK) st = dalloc_t(s, v, nf);
  if (st == MTO_OK) st = dalloc_t(s, &s->partials, partials_count(c));
  if (st == MTO_OK) st = dalloc_t(s, &s->ticket, 4);
  if (st == MTO_OK) st = dalloc_t(s, &s->sc, 1);
  if (st != MTO_OK) return fail(st);
  *out = s;
  return MTO_OK;
}

// Design state and launch shapes of c, for a slot's next solve; a change of
// shape drops the slot's captured graph.
void sync_slot(const mto_ctx* c, mto_ctx* s) {
  bool same = s->tw64 == c->tw64;
  for (int l = 0; l < MAX_LEVELS; ++l) same = same && s->tw[l] == c->tw[l];
  if (!same) {
    invalidate_graphs(s);
    s->tw64 = c->tw64;
    for (int l = 0; l < MAX_LEVELS; ++l) s->tw[l] = c->tw[l];
  }
  s->has_design = c->has_design;
  s->n_phase = c->n_phase;
  s->ph = c->ph;
  s->penal = c->penal;
  s->ipenal = c->ipenal;
}

}  // namespace

namespace mto {

mto_status ensure_slots(mto_ctx* c, int want, int* got) {
  int S = std::max(1, std::min(want, MAX_CONCURRENT_RHS));
  while ((int)c->slots.size() < S - 1) {
    mto_ctx* w = nullptr;
    const mto_status st = make_slot(c, &w);
    if (st == MTO_ERR_OOM) {  // fewer concurrent right-hand sides
      S = (int)c->slots.size() + 1;
      break;
    }
    if (st != MTO_OK) return st;
    c->slots.push_back(w);
  }
  if (S > 1 && !c->ev_slot) CK(cudaEventCreateWithFlags(&c->ev_slot, cudaEventDisableTiming));
  for (int k = 1; k < S; ++k) sync_slot(c, c->slots[k - 1]);
  *got = S;
  return MTO_OK;
}

}  // namespace mto

namespace {

// Enqueues right-hand sides [0, n_rhs) (no host synchronisation): the events
// ev0 / ev1 bracket the device work on the context's stream and the
// right-hand sides' statistics are copied to stats_host (pinned) behind it.
// *S_out is the number of workspaces used (solve_rhs_finish needs it).
mto_status solve_rhs_enqueue(mto_ctx* c, int n_rhs, const double* f_dev, double* u_dev,
                             RhsStats* stats_host, cudaEvent_t ev0, cudaEvent_t ev1, int* S_out) {
  const size_t nd = 2 * (size_t)(c->nelx + 1) * (c->nely + 1);
  c->cs = c->stream;
  const bool polled = c->timing || c->no_while;
  if (!polled) {
    const mto_status b = build_solve_graph(c);
    if (b != MTO_OK) {
      // Conditional graph nodes unavailable: fall back to the polled loop.
      c->no_while = true;
      cudaGetLastError();
    }
  }
  // Right-hand sides at the same time (device-side loop only): right-hand
  // side k runs on workspace k mod S (0: this context), each on its own
  // stream, forked from and joined back into the context's stream.
  int S = 1;
  if (!(c->timing || c->no_while)) {
    ST(ensure_slots(c, std::min(n_rhs, c->o.concurrent_rhs), &S));
    for (int k = 1; k < S; ++k) {
      if (build_solve_graph(c->slots[k - 1]) != MTO_OK) {  // one after another instead
        cudaGetLastError();
        S = k;
        break;
      }
    }
  }
  *S_out = S;
  auto slot_of = [&](int k) { return k % S == 0 ? c : c->slots[k % S - 1]; };
  CK(cudaEventRecord(ev0, c->stream));
  if (S > 1) {
    CK(cudaEventRecord(c->ev_slot, c->stream));
    for (int k = 1; k < S; ++k) CK(cudaStreamWaitEvent(c->slots[k - 1]->stream, c->ev_slot, 0));
  }
  for (int k = 0; k < n_rhs; ++k) {
    mto_ctx* w = slot_of(k);
    w->cs = w->stream;
    ST(enqueue_rhs_prologue(w, f_dev + k * nd, u_dev + k * nd));
    if (c->timing || c->no_while) {
      ST(solve_polled(c));
    } else {
      CK(cudaGraphLaunch(w->solve_exec, w->stream));
      w->launches += w->solve_kernels_fixed;
    }
    ST(enqueue_rhs_epilogue(w, u_dev + k * nd, k));
  }
  for (int k = 1; k < S; ++k) {
    mto_ctx* w = c->slots[k - 1];
    CK(cudaEventRecord(w->ev_slot, w->stream));
    CK(cudaStreamWaitEvent(c->stream, w->ev_slot, 0));
  }
  c->cs = c->stream;
  CK(cudaEventRecord(ev1, c->stream));
  CK(cudaMemcpyAsync(stats_host, c->rhs_stats, sizeof(RhsStats) * n_rhs, cudaMemcpyDeviceToHost,
                     c->stream));
  return MTO_OK;
}

// Statistics of completed right-hand sides (stats_host filled, ms the device
// time of the solve): fills c->last and returns the worst status.
mto_status solve_rhs_finish(mto_ctx* c, int n_rhs, const RhsStats* stats_host, float ms, int S,
                            float ms_setup) {
  auto slot_of = [&](int k) { return k % S == 0 ? c : c->slots[k % S - 1]; };
  mto_status worst = MTO_OK;
  int total = 0;
  for (int k = 0; k < n_rhs; ++k) {
    const RhsStats& r = stats_host[k];
    total += r.iter;
    if (!(c->timing || c->no_while)) {
      // The loop body (two iterations) ran max(1, ceil(iter / 2)) times.
      const long long bodies = r.iter > 0 ? (r.iter + 1) / 2 : 1;
      c->launches += slot_of(k)->body_kernels * bodies;
    }
    const mto_status s = status_of(r);
    if (s != MTO_OK && worst == MTO_OK) worst = s;
  }
  for (mto_ctx* w : c->slots) {
    c->launches += w->launches;
    w->launches = 0;
  }
  const RhsStats& r = stats_host[n_rhs - 1];
  const double fn = std::sqrt(r.ff);
  c->last.iters = total;
  c->last.converged = worst == MTO_OK;
  c->last.rel_res_rec = fn > 0 ? std::sqrt(r.rr) / fn : 0.0;
  c->last.rel_res_true = fn > 0 ? std::sqrt(r.rr_true) / fn : 0.0;
  c->last.ms_solve = ms;
  c->last.ms_setup = ms_setup;
  return worst;
}

// Solves right-hand sides [0, n_rhs) and fills c->last; one host sync.
mto_status solve_rhs(mto_ctx* c, int n_rhs, const double* f_dev, double* u_dev) {
  int S = 1;
  ST(solve_rhs_enqueue(c, n_rhs, f_dev, u_dev, c->rhs_stats_host, c->ev_a, c->ev_b, &S));
  CK(cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev_a, c->ev_b));
  return solve_rhs_finish(c, n_rhs, c->rhs_stats_host, ms, S, c->ms_setup);
}

}  // namespace

// ===========================================================================
// Public API
// ===========================================================================

extern "C" {

void mto_default_opts(mto_solver_opts* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->max_it = 500;
  o->omega = 0.6;
  o->nu1 = 2;
  o->nu2 = 2;
  o->n_coarsen = 3;
  o->coarse_kind = MTO_COARSE_GALERKIN;
  o->precision = MTO_PRECISION_FP64;
  o->rr_every = 25;
  o->flexible = 0;
  o->check_every = 4;
  o->gamma = 1;
  o->concurrent_rhs = 2;
}

const char* mto_cuda_error_string(void) { return cudaGetErrorString(g_last_cuda); }

void mto_set_device_memory_limit(size_t bytes) {
  std::lock_guard<std::mutex> lock(g_mem_mutex);
  g_mem_limit = bytes;
}

size_t mto_device_memory_in_use(void) {
  std::lock_guard<std::mutex> lock(g_mem_mutex);
  return g_mem_in_use;
}

const char* mto_status_string(mto_status s) {
  switch (s) {
    case MTO_OK: return "ok";
    case MTO_ERR_ARG: return "invalid argument";
    case MTO_ERR_UNSUPPORTED_MESH: return "unsupported mesh";
    case MTO_ERR_OOM: return "out of device memory";
    case MTO_ERR_CUDA: return "CUDA error";
    case MTO_ERR_NOT_CONVERGED: return "not converged";
    case MTO_ERR_BREAKDOWN: return "PCG breakdown";
    case MTO_ERR_TIMEOUT: return "device wait timed out";
    case MTO_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

void mto_destroy(mto_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->down) cudaStreamSynchronize(c->down);
  for (mto_ctx* s : c->slots) mto_destroy(s);
  c->slots.clear();
  if (c->ev_slot) cudaEventDestroy(c->ev_slot);
  for (HostCall& h : c->hq) {
    if (h.stats) cudaFreeHost(h.stats);
    if (h.err) cudaFreeHost(h.err);
    for (cudaEvent_t e : {h.setup0, h.setup1, h.t0, h.t1, h.in, h.done})
      if (e) cudaEventDestroy(e);
  }
  for (cudaEvent_t e : {c->ev_stage_free[0], c->ev_stage_free[1], c->ev_u_out, c->ev_g_out, c->ev_cmp})
    if (e) cudaEventDestroy(e);
  if (c->down) cudaStreamDestroy(c->down);
  invalidate_graphs(c);
  for (void* p : c->allocs) device_free(p);
  if (c->sc_host) cudaFreeHost(c->sc_host);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->rhs_stats_host) cudaFreeHost(c->rhs_stats_host);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int d = 0; d < 2; ++d)
        if (c->kev[a][b][d]) cudaEventDestroy(c->kev[a][b][d]);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->ev_a) cudaEventDestroy(c->ev_a);
  if (c->ev_b) cudaEventDestroy(c->ev_b);
  if (c->ev_aux) cudaEventDestroy(c->ev_aux);
  for (cudaEvent_t e : c->ev_chunk)
    if (e) cudaEventDestroy(e);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->fac_stream) cudaStreamDestroy(c->fac_stream);
  if (c->body_stream) cudaStreamDestroy(c->body_stream);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

static mto_status create_impl(mto_ctx* c, int nelx, int nely, double nu, unsigned fixed,
                              const mto_solver_opts& o, int device, void* stream) {
  c->device = device;
  c->nelx = nelx;
  c->nely = nely;
  c->nu = nu;
  c->fixed = fixed;
  c->o = o;
  c->L = o.n_coarsen;
  c->mixed = o.precision == MTO_PRECISION_MIXED;
  c->user_stream = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(device));
  CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking));
  c->cs = c->stream;
  CK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  CK(cudaEventCreate(&c->ev_a));
  CK(cudaEventCreate(&c->ev_b));
  CK(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&c->fac_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_aux, cudaEventDisableTiming));
  for (cudaEvent_t& e : c->ev_chunk) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CK(cudaMallocHost(&c->sc_host, sizeof(DevScalars)));
  CK(cudaMallocHost(&c->err_host, sizeof(int)));
  CK(cudaMallocHost(&c->rhs_stats_host, sizeof(RhsStats) * MAX_RHS));

  // Element-operator constants (plane stress, Eq. 8; strain basis, mto_common.cuh).
  const double kap = 1.0 / (4.0 * (1.0 - nu * nu)), gs = 0.5 * (1.0 - nu);
  c->kf64 = {kap, kap * nu, kap * (1.0 + gs) / 3.0, kap * gs};
  c->kf32 = {(float)c->kf64.kA, (float)c->kf64.kB, (float)c->kf64.kC, (float)c->kf64.kG};
  const double kdiag = kap * (1.0 + (1.0 + gs) / 3.0 + gs);  // KE_00 at E = 1
  c->w_over_kdiag = o.omega / kdiag;

  if (c->L + 1 > MAX_LEVELS) return MTO_ERR_UNSUPPORTED_MESH;
  c->lv.resize(c->L + 1);
  for (int l = 0; l <= c->L; ++l) {
    const int sh = c->L - l;
    c->lv[l].g = make_grid(nelx >> sh, nely >> sh, fixed);
  }
  const size_t vsz = c->mixed ? sizeof(float2) : sizeof(double2);
  const size_t csz = c->mixed ? sizeof(float) : sizeof(double);
  for (int l = 0; l <= c->L; ++l) {
    LevelBuf& B = c->lv[l];
    const size_t n = (size_t)B.g.size();
    ST(dalloc(c, &B.z[0], n * vsz));
    ST(dalloc(c, &B.z[1], n * vsz));
    if (l < c->L) {
      ST(dalloc(c, &B.b, n * vsz));
      ST(dalloc(c, &B.coef, n * NCOEF * csz));
      ST(dalloc(c, &B.invd2, n * vsz));
      ST(dalloc_t(c, &B.mom, n * NMOM));
    }
    if (l == 0) ST(dalloc_t(c, &B.coef64, n * NCOEF));
  }
  const Grid& gf = c->lv[c->L].g;
  const size_t nf = (size_t)gf.size();
  ST(dalloc_t(c, &c->E64, nf));
  ST(dalloc_t(c, &c->Ek4, 4 * nf));
  if (c->mixed) {
    ST(dalloc_t(c, &c->Ebf, nf));
    ST(dalloc_t(c, &c->r32, nf));
  } else {
    ST(dalloc_t(c, &c->invd1, nf));
  }
  ST(dalloc_t(c, &c->x, nf));
  ST(dalloc_t(c, &c->r, nf));
  if (c->mixed) ST(dalloc_t(c, &c->r_alt, nf));
  ST(dalloc_t(c, &c->q, nf));
  ST(dalloc_t(c, &c->f, nf));
  ST(dalloc_t(c, &c->tmp, nf));
  ST(dalloc_t(c, &c->p[0], nf));
  ST(dalloc_t(c, &c->p[1], nf));

  // Coarsest grid: free-DOF numbering (row-major over nodes, u_x before u_y),
  // its inverse map, and the half bandwidth of K_0 in that numbering.
  const Grid& g0 = c->lv[0].g;
  std::vector<int> idx(2 * (size_t)g0.size() + 1, -1);
  std::vector<int> inv;
  for (int j = 0; j <= g0.ny; ++j)
    for (int i = 0; i <= g0.nx; ++i)
      if (!g0.is_fixed(i, j))
        for (int comp = 0; comp < 2; ++comp) {
          idx[2 * g0.at(i, j) + comp] = (int)inv.size();
          inv.push_back((int)(2 * g0.at(i, j) + comp));
        }
  c->n0 = (int)inv.size();
  if (c->n0 > GEMV_MAXN) return MTO_ERR_UNSUPPORTED_MESH;
  int bw = 0;
  for (int j = 0; j <= g0.ny; ++j)
    for (int i = 0; i <= g0.nx; ++i)
      for (int comp = 0; comp < 2; ++comp) {
        const int a = idx[2 * g0.at(i, j) + comp];
        if (a < 0) continue;
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            if (!g0.valid(i + di, j + dj)) continue;
            for (int c2 = 0; c2 < 2; ++c2) {
              const int b = idx[2 * g0.at(i + di, j + dj) + c2];
              if (b >= 0 && std::abs(a - b) > bw) bw = std::abs(a - b);
            }
          }
      }
  c->bw0 = bw;
  // The factorisation keeps the (i, j) index pairs of a band triangle in
  // shared memory (2 bw (bw + 1) bytes).
  if (bw > MAX_COARSEST_BW) return MTO_ERR_UNSUPPORTED_MESH;
  std::vector<int> dof(2 * (size_t)g0.size() + c->n0);
  std::memcpy(dof.data(), idx.data(), sizeof(int) * 2 * (size_t)g0.size());
  std::memcpy(dof.data() + 2 * (size_t)g0.size(), inv.data(), sizeof(int) * c->n0);
  ST(dalloc_t(c, &c->dof_index, dof.size()));
  CK(cudaMemcpy(c->dof_index, dof.data(), sizeof(int) * dof.size(), cudaMemcpyHostToDevice));
  ST(dalloc_t(c, &c->Kd, (size_t)c->n0 * (c->bw0 + 1)));
  ST(dalloc_t(c, &c->invL, (size_t)c->n0));
  ST(dalloc_t(c, &c->Lsc, 2 * (size_t)c->n0 * (c->bw0 + 1)));
  ST(dalloc_t(c, &c->Kinv, (size_t)c->n0 * c->n0));
  ST(dalloc_t(c, &c->err_flag, 1));

  ST(dalloc_t(c, &c->partials, partials_count(c)));
  ST(dalloc_t(c, &c->ticket, 4));
  ST(dalloc_t(c, &c->sc, 1));
  ST(dalloc_t(c, &c->rhs_stats, MAX_RHS));
  // Opt-in shared memory of the coarsest factorisation, set once here so that
  // set_design can be captured into graphs.
  CK(prepare_cholesky_inverse(c->n0, c->bw0));
  CK(prepare_coarsest_gemv(c->n0));
  return MTO_OK;
}

mto_status mto_create_mesh(mto_ctx** out, int nelx, int nely, double nu, unsigned fixed_edges,
                           const mto_solver_opts* opts, int device, void* cuda_stream) {
  NvtxRange nvtx_range("mto_create_mesh");
  if (!out) return MTO_ERR_ARG;
  *out = nullptr;
  mto_solver_opts o;
  mto_default_opts(&o);
  if (opts) o = *opts;
  if (nelx < 1 || nely < 1 || !(nu > -1.0 && nu < 0.5) || fixed_edges == 0u || fixed_edges > 15u ||
      !valid_opts(o) || device < 0)
    return MTO_ERR_ARG;
  if (nelx % (1 << o.n_coarsen) || nely % (1 << o.n_coarsen)) return MTO_ERR_UNSUPPORTED_MESH;
  if ((long long)nelx * nely > (1LL << 30)) return MTO_ERR_UNSUPPORTED_MESH;
  mto_ctx* c = new (std::nothrow) mto_ctx();
  if (!c) return MTO_ERR_OOM;
  mto_status s = create_impl(c, nelx, nely, nu, fixed_edges, o, device, cuda_stream);
  if (s != MTO_OK) {
    cudaGetLastError();
    mto_destroy(c);
    return s;
  }
  *out = c;
  return MTO_OK;
}

static bool valid_design(int n_phase, const double* E_phase, double penal) {
  if (!E_phase || n_phase < 1 || n_phase > 16 || !(penal >= 1.0 && penal <= 64.0)) return false;
  for (int i = 0; i < n_phase; ++i)
    if (!(E_phase[i] > 0.0 && E_phase[i] < 1e300)) return false;
  return true;
}

mto_status mto_set_design(mto_ctx* c, int n_phase, const double* x_dev, const double* E_phase,
                          double penal) {
  NvtxRange nvtx_range("mto_set_design");
  if (!c || !x_dev || !valid_design(n_phase, E_phase, penal)) return MTO_ERR_ARG;
  ST(enter(c));
  c->has_design = false;
  mto_status s = set_design_sync(c, n_phase, x_dev, E_phase, penal);
  mto_status s2 = leave(c);
  return s != MTO_OK ? s : s2;
}

mto_status mto_solve(mto_ctx* c, int n_rhs, const double* f_dev, double* u_dev,
                     mto_solve_stats* stats) {
  NvtxRange nvtx_range("mto_solve");
  if (!c || n_rhs < 1 || n_rhs > MAX_RHS || !f_dev || !u_dev || !aligned16(f_dev) || !aligned16(u_dev))
    return MTO_ERR_ARG;
  if (!c->has_design) return MTO_ERR_STATE;
  ST(enter(c));
  const mto_status s = solve_rhs(c, n_rhs, f_dev, u_dev);
  if (s == MTO_ERR_CUDA || s == MTO_ERR_OOM || s == MTO_ERR_STATE) {
    leave(c);
    return s;
  }
  ST(leave(c));
  if (stats) *stats = c->last;
  return s;
}

mto_status mto_last_stats(mto_ctx* c, mto_solve_stats* stats) {
  if (!c || !stats) return MTO_ERR_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->stream));
  *stats = c->last;
  return MTO_OK;
}

mto_status mto_compliance_grad(mto_ctx* c, int n_rhs, const double* f_dev, const double* u_dev,
                               double* compliance_dev, double* dcdx_dev) {
  NvtxRange nvtx_range("mto_compliance_grad");
  if (!c || n_rhs < 1 || !f_dev || !u_dev || !compliance_dev || !aligned16(f_dev) || !aligned16(u_dev))
    return MTO_ERR_ARG;
  if (!c->has_design) return MTO_ERR_STATE;
  ST(enter(c));
  ST(enqueue_compliance(c, n_rhs, f_dev, u_dev, compliance_dev, dcdx_dev));
  return leave(c);
}

mto_status mto_run_host(mto_ctx* c, int n_phase, const double* x_host, const double* E_phase,
                        double penal, int n_rhs, const double* f_host, double* u_host,
                        double* compliance_host, double* dcdx_host, mto_solve_stats* stats) {
  NvtxRange nvtx_range("mto_run_host");
  if (!c || !x_host || n_rhs < 1 || n_rhs > MAX_RHS || !f_host || !u_host || !compliance_host ||
      !valid_design(n_phase, E_phase, penal))
    return MTO_ERR_ARG;
  if (c->hq_count > 0) return MTO_ERR_STATE;  // pipelined calls still in flight
  const size_t nel = (size_t)c->nelx * c->nely;
  const size_t nd = 2 * (size_t)(c->nelx + 1) * (c->nely + 1);
  ST(grow(c, &c->xdes, &c->xdes_cap, (size_t)n_phase * nel));
  ST(grow(c, &c->hf, &c->hf_cap, (size_t)n_rhs * nd));
  ST(grow(c, &c->hu, &c->hu_cap, (size_t)n_rhs * nd));
  size_t ccap = (size_t)c->hc_cap;
  ST(grow(c, &c->hc, &ccap, (size_t)n_rhs));
  c->hc_cap = (int)ccap;
  if (dcdx_host) ST(grow(c, &c->hg, &c->hg_cap, (size_t)n_phase * nel));
  ST(enter(c));
  c->has_design = false;
  c->cs = c->stream;
  const int nch = std::min(HOST_CHUNKS, c->nely);
  auto rows = [&](int k) { return (int)((long long)c->nely * k / nch); };
  // The side stream starts after all earlier work of the compute stream.
  CK(cudaEventRecord(c->ev_aux, c->stream));
  CK(cudaStreamWaitEvent(c->aux, c->ev_aux, 0));
  // Design: x arrives in row chunks on the side stream and the moduli of a
  // chunk are formed while the next one is in flight; f and the zero start
  // follow on the side stream while the coarse hierarchy is built.
  CK(cudaEventRecord(c->ev_a, c->stream));
  design_params(c, n_phase, E_phase, penal);
  for (int k = 0; k < nch; ++k) {
    const int j0 = rows(k), j1 = rows(k + 1);
    for (int p = 0; p < n_phase; ++p) {
      const size_t off = (size_t)p * nel + (size_t)j0 * c->nelx;
      CK(cudaMemcpyAsync(c->xdes + off, x_host + off, sizeof(double) * (size_t)(j1 - j0) * c->nelx,
                         cudaMemcpyHostToDevice, c->aux));
    }
    CK(cudaEventRecord(c->ev_chunk[k], c->aux));
    CK(cudaStreamWaitEvent(c->stream, c->ev_chunk[k], 0));
    ST(enqueue_modulus(c, j0, j1));
  }
  CK(cudaMemcpyAsync(c->hf, f_host, sizeof(double) * n_rhs * nd, cudaMemcpyHostToDevice, c->aux));
  CK(cudaMemsetAsync(c->hu, 0, sizeof(double) * n_rhs * nd, c->aux));
  CK(cudaEventRecord(c->ev_aux, c->aux));
  ST(enqueue_hierarchy(c));
  CK(cudaMemcpyAsync(c->err_host, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaEventRecord(c->ev_b, c->stream));
  CK(cudaStreamWaitEvent(c->stream, c->ev_aux, 0));  // f and u have landed
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaEventElapsedTime(&c->ms_setup, c->ev_a, c->ev_b));
  if (*c->err_host) {
    leave(c);
    return MTO_ERR_BREAKDOWN;
  }
  c->has_design = true;
  const mto_status s = solve_rhs(c, n_rhs, c->hf, c->hu);
  if (s == MTO_ERR_CUDA || s == MTO_ERR_OOM || s == MTO_ERR_STATE) return s;
  c->cs = c->stream;
  // Results: u leaves on the side stream while the compliance and the
  // sensitivities are formed; the sensitivities leave in row chunks.
  CK(cudaEventRecord(c->ev_aux, c->stream));
  CK(cudaStreamWaitEvent(c->aux, c->ev_aux, 0));
  CK(cudaMemcpyAsync(u_host, c->hu, sizeof(double) * n_rhs * nd, cudaMemcpyDeviceToHost, c->aux));
  ST(enqueue_compliance(c, n_rhs, c->hf, c->hu, c->hc, nullptr));
  CK(cudaMemcpyAsync(compliance_host, c->hc, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, c->stream));
  if (dcdx_host) {
    const long long nn = (long long)(c->nelx + 1) * (c->nely + 1);
    for (int k = 0; k < nch; ++k) {
      for (int r = 0; r < n_rhs; ++r)
        KL(launch_sensitivity(c->nelx, c->nely, c->n_phase, c->xdes, c->ph, c->penal, c->ipenal,
                              c->kf64, c->hu + 2 * nn * r, c->hg, r > 0, c->stream, c->num_sms,
                              rows(k), rows(k + 1)));
      CK(cudaEventRecord(c->ev_chunk[k], c->stream));
    }
    // Issued after every launch: a copy to pageable memory returns only
    // when it is done.
    for (int k = 0; k < nch; ++k) {
      CK(cudaStreamWaitEvent(c->aux, c->ev_chunk[k], 0));
      const int j0 = rows(k), j1 = rows(k + 1);
      for (int p = 0; p < n_phase; ++p) {
        const size_t off = (size_t)p * nel + (size_t)j0 * c->nelx;
        CK(cudaMemcpyAsync(dcdx_host + off, c->hg + off, sizeof(double) * (size_t)(j1 - j0) * c->nelx,
                           cudaMemcpyDeviceToHost, c->aux));
      }
    }
  }
  CK(cudaStreamSynchronize(c->aux));
  CK(cudaStreamSynchronize(c->stream));
  ST(leave(c));
  if (stats) *stats = c->last;
  return s;
}

// Streams, pinned records and events of the pipelined host calls, created on
// first use (what an earlier failed attempt already created is kept; all of
// it is released by mto_destroy).
static mto_status hq_setup(mto_ctx* c) {
  if (c->hq_ready) return MTO_OK;
  if (!c->down) CK(cudaStreamCreateWithFlags(&c->down, cudaStreamNonBlocking));
  for (HostCall& h : c->hq) {
    if (!h.stats) CK(cudaMallocHost(&h.stats, sizeof(RhsStats) * MAX_RHS));
    if (!h.err) CK(cudaMallocHost(&h.err, sizeof(int)));
    for (cudaEvent_t* e : {&h.setup0, &h.setup1, &h.t0, &h.t1})
      if (!*e) CK(cudaEventCreate(e));
    for (cudaEvent_t* e : {&h.in, &h.done})
      if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  for (cudaEvent_t* e : {&c->ev_stage_free[0], &c->ev_stage_free[1], &c->ev_u_out, &c->ev_g_out, &c->ev_cmp})
    if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  c->hq_ready = true;
  return MTO_OK;
}

mto_status mto_run_host_async(mto_ctx* c, int n_phase, const double* x_host, const double* E_phase,
                              double penal, int n_rhs, const double* f_host, double* u_host,
                              double* compliance_host, double* dcdx_host) {
  NvtxRange nvtx_range("mto_run_host_async");
  if (!c || !x_host || n_rhs < 1 || n_rhs > MAX_RHS || !f_host || !u_host || !compliance_host ||
      !valid_design(n_phase, E_phase, penal))
    return MTO_ERR_ARG;
  if (c->timing || c->hq_count >= 2) return MTO_ERR_STATE;
  const size_t nel = (size_t)c->nelx * c->nely;
  const size_t nd = 2 * (size_t)(c->nelx + 1) * (c->nely + 1);
  ST(enter(c));
  ST(hq_setup(c));
  const int slot = (c->hq_head + c->hq_count) & 1;
  HostCall& h = c->hq[slot];
  // Buffers (grown ones keep their old allocation alive for a call in flight).
  // Both staging areas grow together, so that the allocation, which can wait
  // for the device, happens before this call enqueues anything rather than
  // behind the previous call's kernels.
  ST(grow(c, &c->xdes, &c->xdes_cap, (size_t)n_phase * nel));
  for (int s = 0; s < 2; ++s) {
    ST(grow(c, &c->xstage[s], &c->xstage_cap[s], (size_t)n_phase * nel));
    ST(grow(c, &c->fstage[s], &c->fstage_cap[s], (size_t)n_rhs * nd));
  }
  ST(grow(c, &c->hu, &c->hu_cap, (size_t)n_rhs * nd));
  size_t ccap = (size_t)c->hc_cap;
  ST(grow(c, &c->hc, &ccap, (size_t)n_rhs));
  c->hc_cap = (int)ccap;
  if (dcdx_host) ST(grow(c, &c->hg, &c->hg_cap, (size_t)n_phase * nel));
  double* xs = c->xstage[slot];
  double* fs = c->fstage[slot];
  double *hu = c->hu, *hc = c->hc, *hg = c->hg;
  c->cs = c->stream;
  // Upload (side stream): once the call that last used this staging slot has
  // consumed its inputs.
  CK(cudaStreamWaitEvent(c->aux, c->ev_stage_free[slot], 0));
  CK(cudaMemcpyAsync(xs, x_host, sizeof(double) * n_phase * nel, cudaMemcpyHostToDevice, c->aux));
  CK(cudaMemcpyAsync(fs, f_host, sizeof(double) * n_rhs * nd, cudaMemcpyHostToDevice, c->aux));
  CK(cudaEventRecord(h.in, c->aux));
  // Design (compute stream, after the previous call's compute).
  CK(cudaStreamWaitEvent(c->stream, h.in, 0));
  CK(cudaEventRecord(h.setup0, c->stream));
  CK(cudaMemcpyAsync(c->xdes, xs, sizeof(double) * n_phase * nel, cudaMemcpyDeviceToDevice, c->stream));
  design_params(c, n_phase, E_phase, penal);
  ST(enqueue_modulus(c, 0, c->nely));
  ST(enqueue_hierarchy(c));
  CK(cudaMemcpyAsync(h.err, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaEventRecord(h.setup1, c->stream));
  c->has_design = true;
  // Solve from zero into hu, once the previous call's u has left.
  CK(cudaStreamWaitEvent(c->stream, c->ev_u_out, 0));
  CK(cudaMemsetAsync(hu, 0, sizeof(double) * n_rhs * nd, c->stream));
  int S = 1;
  ST(solve_rhs_enqueue(c, n_rhs, fs, hu, h.stats, h.t0, h.t1, &S));
  c->cs = c->stream;
  // Compliance and sensitivities, once the previous call's results have left.
  CK(cudaStreamWaitEvent(c->stream, c->ev_g_out, 0));
  ST(enqueue_compliance(c, n_rhs, fs, hu, hc, nullptr));
  CK(cudaEventRecord(c->ev_cmp, c->stream));
  const int nch = std::min(HOST_CHUNKS, c->nely);
  auto rows = [&](int k) { return (int)((long long)c->nely * k / nch); };
  if (dcdx_host) {
    const long long nn = (long long)(c->nelx + 1) * (c->nely + 1);
    for (int k = 0; k < nch; ++k) {
      for (int r = 0; r < n_rhs; ++r)
        KL(launch_sensitivity(c->nelx, c->nely, c->n_phase, c->xdes, c->ph, c->penal, c->ipenal,
                              c->kf64, hu + 2 * nn * r, hg, r > 0, c->stream, c->num_sms, rows(k),
                              rows(k + 1)));
      CK(cudaEventRecord(c->ev_chunk[k], c->stream));
    }
  }
  CK(cudaEventRecord(c->ev_stage_free[slot], c->stream));
  // Download (own stream).
  CK(cudaStreamWaitEvent(c->down, c->ev_cmp, 0));
  CK(cudaMemcpyAsync(u_host, hu, sizeof(double) * n_rhs * nd, cudaMemcpyDeviceToHost, c->down));
  CK(cudaEventRecord(c->ev_u_out, c->down));
  CK(cudaMemcpyAsync(compliance_host, hc, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, c->down));
  if (dcdx_host) {
    for (int k = 0; k < nch; ++k) {
      CK(cudaStreamWaitEvent(c->down, c->ev_chunk[k], 0));
      const int j0 = rows(k), j1 = rows(k + 1);
      for (int p = 0; p < n_phase; ++p) {
        const size_t off = (size_t)p * nel + (size_t)j0 * c->nelx;
        CK(cudaMemcpyAsync(dcdx_host + off, hg + off, sizeof(double) * (size_t)(j1 - j0) * c->nelx,
                           cudaMemcpyDeviceToHost, c->down));
      }
    }
  }
  CK(cudaEventRecord(c->ev_g_out, c->down));
  CK(cudaEventRecord(h.done, c->down));
  h.n_rhs = n_rhs;
  h.S = S;
  h.u_host = u_host;
  h.c_host = compliance_host;
  h.g_host = dcdx_host;
  c->hq_count += 1;
  return leave(c);
}

mto_status mto_run_host_wait(mto_ctx* c, mto_solve_stats* stats) {
  NvtxRange nvtx_range("mto_run_host_wait");
  if (!c) return MTO_ERR_ARG;
  if (c->hq_count == 0) return MTO_ERR_STATE;
  CK(cudaSetDevice(c->device));
  HostCall& h = c->hq[c->hq_head];
  CK(cudaEventSynchronize(h.done));
  c->hq_head ^= 1;
  c->hq_count -= 1;
  float ms = 0.f, ms_setup = 0.f;
  CK(cudaEventElapsedTime(&ms, h.t0, h.t1));
  CK(cudaEventElapsedTime(&ms_setup, h.setup0, h.setup1));
  if (*h.err) {
    if (c->hq_count == 0) c->has_design = false;  // unless a later call replaced the design
    return MTO_ERR_BREAKDOWN;
  }
  const mto_status s = solve_rhs_finish(c, h.n_rhs, h.stats, ms, h.S, ms_setup);
  if (stats) *stats = c->last;
  return s;
}

mto_status mto_apply_operator(mto_ctx* c, int level, int use_vcycle_operator, const double* v_dev,
                              double* y_dev) {
  if (!c || !v_dev || !y_dev || level < 0 || level > c->L || !aligned16(v_dev) || !aligned16(y_dev))
    return MTO_ERR_ARG;
  if (!c->has_design) return MTO_ERR_STATE;
  ST(enter(c));
  LevelBuf& B = c->lv[level];
  const int tw = target_warps(c, level);
  const bool fine = level == c->L;
  if (fine && (!c->mixed || !use_vcycle_operator)) {
    KL(launch_pack(B.g, v_dev, c->tmp, c->cs, c->num_sms));
    SweepParams<double> p = base_params<double>(c, B.g);
    p.v = c->tmp;
    p.out = c->q;
    p.E = c->Ek4;
    KL(launch_sweep<double>(SRC_FINE64, MODE_APPLY, false, false, p,
                            tw, c->num_sms, c->cs));
    KL(launch_unpack(B.g, c->q, y_dev, c->cs, c->num_sms));
  } else if (c->mixed && level > 0) {
    KL(launch_pack_f32(B.g, v_dev, (float2*)B.z[0], c->cs, c->num_sms));
    SweepParams<float> p = base_params<float>(c, B.g);
    p.v = (const float2*)B.z[0];
    p.out = (float2*)B.z[1];
    p.E = c->Ebf;
    p.kf = c->kf32;
    p.coef = (const float*)B.coef;
    set_cmom(c, p);
    const bool cfine = level == c->L - 1;
    if (cfine) set_cfine(c, p);
    KL(launch_sweep<float>(fine ? SRC_FINEBF : (cfine ? SRC_CFINE : SRC_CMOM), MODE_APPLY, false,
                           false, p, tw, c->num_sms, c->cs));
    KL(launch_unpack_f32(B.g, (const float2*)B.z[1], y_dev, c->cs, c->num_sms));
  } else {
    // float64 coarse levels.  The mixed cycle's coarsest level is float64
    // too; its level vectors are float2, so the finest level's float64
    // scratch vectors (larger than any coarse grid) hold the operands.
    double2* vin = c->mixed ? c->tmp : (double2*)B.z[0];
    double2* vout = c->mixed ? c->q : (double2*)B.z[1];
    KL(launch_pack(B.g, v_dev, vin, c->cs, c->num_sms));
    SweepParams<double> p = base_params<double>(c, B.g);
    p.v = vin;
    p.out = vout;
    p.coef = c->mixed ? B.coef64 : (const double*)B.coef;
    KL(launch_sweep<double>(SRC_COARSE, MODE_APPLY, false, false, p,
                            tw, c->num_sms, c->cs));
    KL(launch_unpack(B.g, vout, y_dev, c->cs, c->num_sms));
  }
  return leave(c);
}

mto_status mto_apply_preconditioner(mto_ctx* c, const double* r_dev, double* z_dev) {
  if (!c || !r_dev || !z_dev || !aligned16(r_dev) || !aligned16(z_dev)) return MTO_ERR_ARG;
  if (!c->has_design) return MTO_ERR_STATE;
  ST(enter(c));
  LevelBuf& B = c->lv[c->L];
  KL(launch_pack(B.g, r_dev, c->r, c->cs, c->num_sms));
  int zi = 0;
  if (c->mixed) {
    KL(launch_pack_f32(B.g, r_dev, c->r32, c->cs, c->num_sms));
    ST(fine_cycle<float>(c, nullptr, false, &zi));
    KL(launch_unpack_f32(B.g, (const float2*)B.z[zi], z_dev, c->cs, c->num_sms));
  } else {
    ST(fine_cycle<double>(c, nullptr, false, &zi));
    KL(launch_unpack(B.g, (const double2*)B.z[zi], z_dev, c->cs, c->num_sms));
  }
  return leave(c);
}

mto_status mto_get_info(mto_ctx* c, int* n_levels, int* coarsest_free_dofs) {
  if (!c) return MTO_ERR_ARG;
  if (n_levels) *n_levels = c->L + 1;
  if (coarsest_free_dofs) *coarsest_free_dofs = c->n0;
  return MTO_OK;
}

mto_status mto_get_moduli(mto_ctx* c, double* E_dev) {
  if (!c || !E_dev) return MTO_ERR_ARG;
  if (!c->has_design) return MTO_ERR_STATE;
  ST(enter(c));
  KL(launch_unpack_elems(c->lv[c->L].g, c->E64, E_dev, c->cs, c->num_sms));
  return leave(c);
}

mto_status mto_set_kernel_timing(mto_ctx* c, int enable) {
  if (!c) return MTO_ERR_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->cs));
  if (enable && !c->kev[0][0][0])
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int d = 0; d < 2; ++d) CK(cudaEventCreate(&c->kev[a][b][d]));
  if ((bool)enable != c->timing) invalidate_graphs(c);
  c->timing = enable != 0;
  c->ksum[0] = c->ksum[1] = 0.0;
  c->kcnt[0] = c->kcnt[1] = 0;
  return MTO_OK;
}

mto_status mto_get_kernel_times(mto_ctx* c, double* ms_avg, long long* samples) {
  if (!c || !ms_avg || !samples) return MTO_ERR_ARG;
  for (int k = 0; k < 2; ++k) {
    samples[k] = c->kcnt[k];
    ms_avg[k] = c->kcnt[k] ? c->ksum[k] / (double)c->kcnt[k] : 0.0;
  }
  return MTO_OK;
}

mto_status mto_get_launch_count(mto_ctx* c, long long* launches) {
  if (!c || !launches) return MTO_ERR_ARG;
  *launches = c->launches;
  return MTO_OK;
}

}  // extern "C"
