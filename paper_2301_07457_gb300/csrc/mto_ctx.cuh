// Internal definition of the libmto context, shared by the translation units
// that enqueue its work (mto_api.cu: single solves and the C ABI;
// mto_batch.cu: batched graphs and the launch-shape tuner).
#pragma once

#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mto.h"
#include "mto_launch.h"

namespace mto {

struct LevelBuf {
  Grid g{};
  void* z[2] = {nullptr, nullptr};  // V2<T> vectors (ping-pong)
  void* b = nullptr;                // right-hand side of this level
  void* coef = nullptr;             // T coefficients, NCOEF * g.size()
  void* invd2 = nullptr;            // V2<T> w / D
  double* mom = nullptr;            // NMOM * g.size() (coarse levels)
  double* coef64 = nullptr;         // level 0: float64 coefficients for the dense matrix
};

constexpr int MAX_LEVELS = 16;
constexpr int MAX_RHS = 64;
// Right-hand sides of one mto_solve solved at the same time (opts.concurrent_rhs).
constexpr int MAX_CONCURRENT_RHS = 4;
// Launch shapes: warps a sweep exposes, per SM (upper end of the tuner's
// range).  Target 0 means one full wave of the kernel: its resident blocks
// per SM times the SM count (the default).
constexpr int MAX_TARGET_WARPS_PER_SM = 128;

// Row chunks in which mto_run_host moves x in and dC/dx out, each chunk's
// transfer overlapping the kernels of its neighbours.
constexpr int HOST_CHUNKS = 4;

// One pipelined host call (mto_run_host_async) in flight: where its results
// go, its statistics and the events that mark its progress.
struct HostCall {
  int n_rhs = 0, S = 1;
  double *u_host = nullptr, *c_host = nullptr, *g_host = nullptr;
  RhsStats* stats = nullptr;  // pinned [MAX_RHS]
  int* err = nullptr;         // pinned: the design's factorisation failed
  cudaEvent_t setup0 = nullptr, setup1 = nullptr, t0 = nullptr, t1 = nullptr;
  cudaEvent_t in = nullptr;    // inputs staged on the device
  cudaEvent_t done = nullptr;  // results in host memory
};

}  // namespace mto

struct mto_ctx {
  int device = 0, num_sms = 1;
  cudaStream_t user_stream = nullptr, stream = nullptr;
  // Stream that the enqueue functions use: `stream`, or the stream that
  // captures the body of the solver's device-side loop.
  cudaStream_t cs = nullptr, body_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_a = nullptr, ev_b = nullptr;
  // Side stream of set_design: the coarsest factor and inverse, joined back
  // before the call's work ends.
  cudaStream_t fac_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // Side stream of mto_run_host: host transfers that overlap the compute stream.
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_aux = nullptr;
  cudaEvent_t ev_chunk[mto::HOST_CHUNKS] = {};
  int nelx = 0, nely = 0;
  double nu = 0.3;
  unsigned fixed = 0;
  mto_solver_opts o{};
  int L = 0;
  bool mixed = false;
  std::vector<mto::LevelBuf> lv;
  // finest level
  double* E64 = nullptr;
  double* Ek4 = nullptr;  // E (kA, kB, kC, kG) per element, for the float64 sweeps
  __nv_bfloat16* Ebf = nullptr;
  double* invd1 = nullptr;
  double2 *x = nullptr, *r = nullptr, *q = nullptr, *f = nullptr, *tmp = nullptr;
  double2* p[2] = {nullptr, nullptr};
  float2* r32 = nullptr;
  // Mixed precision: the PCG step of parity par keeps r in (par ? r_alt : r).
  // The first smoothing sweep applies the update r -= alpha q out of place,
  // since neighbouring warps still read the old r on their halo rows.
  double2* r_alt = nullptr;
  // coarsest grid
  int n0 = 0, bw0 = 0;
  int* dof_index = nullptr;
  double *Kd = nullptr, *Kinv = nullptr, *invL = nullptr;  // Kd: band storage of K_0 / its factor
  double* Lsc = nullptr;  // the factor scaled by its columns' and rows' pivots (inverse)
  int* err_flag = nullptr;
  // reductions
  double* partials = nullptr;
  unsigned* ticket = nullptr;
  mto::DevScalars* sc = nullptr;
  mto::DevScalars* sc_host = nullptr;  // pinned
  int* err_host = nullptr;             // pinned
  mto::RhsStats* rhs_stats = nullptr;       // device [MAX_RHS]
  mto::RhsStats* rhs_stats_host = nullptr;  // pinned [MAX_RHS]
  // design
  bool has_design = false;
  int n_phase = 0;
  mto::PhaseTable ph{};
  double penal = 3.0;
  int ipenal = 3;
  double* xdes = nullptr;
  size_t xdes_cap = 0;
  // host-call staging (mto_run_host)
  double *hf = nullptr, *hu = nullptr, *hc = nullptr, *hg = nullptr;
  size_t hf_cap = 0, hu_cap = 0, hg_cap = 0;
  int hc_cap = 0;
  // graph of two PCG iterations (host-polled loop, used when kernel timing is on)
  cudaGraphExec_t gexec = nullptr;
  long long graph_kernels = 0;  // kernel nodes in that graph
  // graph of a whole solve with a device-side loop (conditional while node)
  cudaGraphExec_t solve_exec = nullptr;
  long long solve_kernels_fixed = 0;  // kernels outside the loop body
  long long body_kernels = 0;         // kernels of one loop body (two iterations)
  long long launches = 0;             // kernels launched by this context (graph nodes included)
  // launch shapes: target warps of the V-cycle sweeps per level and of the
  // float64 outer sweeps (K p, residuals) on the finest level (0 = one full
  // wave of the kernel), set by the tuner
  int tw[mto::MAX_LEVELS] = {};
  int tw64 = 0;
  // optional event pairs around the hot kernels of each graph iteration:
  // [parity][0 = outer K p sweep, 1 = first finest-level smoothing sweep][start, end]
  bool timing = false;
  bool no_while = false;  // the device-side loop could not be built: host-polled loop
  cudaEvent_t kev[2][2][2] = {};
  double ksum[2] = {0.0, 0.0};
  long long kcnt[2] = {0, 0};
  int cur_par = -1;
  // constants
  mto::FineConst<double> kf64{};
  mto::FineConst<float> kf32{};
  double w_over_kdiag = 0.0;
  // stats
  float ms_setup = 0.f;
  mto_solve_stats last{};
  std::vector<void*> allocs;
  // Concurrent right-hand sides: workspaces that share this context's design
  // data (moduli, smoother diagonals, coarse operators, coarsest inverse) and
  // own the solve's vectors, scalars, streams and solve graph.  Created on the
  // first solve with two or more right-hand sides; `parent` is set in them.
  std::vector<mto_ctx*> slots;
  mto_ctx* parent = nullptr;
  cudaEvent_t ev_slot = nullptr;
  // Pipelined host calls: at most two in flight, in queue order from
  // hq_head.  Inputs are staged in two device buffers (the call's slot), so
  // that a call's upload overlaps the previous call's solve; results leave
  // on their own stream, overlapping the next call.
  mto::HostCall hq[2];
  int hq_head = 0, hq_count = 0;
  bool hq_ready = false;  // events, pinned buffers and the download stream exist
  cudaStream_t down = nullptr;
  double* xstage[2] = {nullptr, nullptr};
  double* fstage[2] = {nullptr, nullptr};
  size_t xstage_cap[2] = {0, 0}, fstage_cap[2] = {0, 0};
  cudaEvent_t ev_stage_free[2] = {nullptr, nullptr};  // the slot's staged inputs are consumed
  cudaEvent_t ev_u_out = nullptr, ev_g_out = nullptr, ev_cmp = nullptr;
};

namespace mto {

// Last CUDA error that made a call of this thread return MTO_ERR_CUDA.
extern thread_local cudaError_t g_last_cuda;

#define CK(call)                    \
  do {                              \
    cudaError_t e_ = (call);        \
    if (e_ != cudaSuccess) {        \
      ::mto::g_last_cuda = e_;      \
      return MTO_ERR_CUDA;          \
    }                               \
  } while (0)

// A kernel launch made by the context: counted, then checked.
#define KL(call)              \
  do {                        \
    c->launches += 1;         \
    CK(call);                 \
  } while (0)

#define ST(call)                          \
  do {                                    \
    mto_status s_ = (call);               \
    if (s_ != MTO_OK) return s_;          \
  } while (0)

// Device memory of the library: every allocation goes through these, which
// keep a process-wide count of the bytes held and refuse an allocation that
// would pass the limit set by mto_set_device_memory_limit (0: none) with
// cudaErrorMemoryAllocation, without calling cudaMalloc.
cudaError_t device_alloc(void** p, size_t bytes);
void device_free(void* p);

// Nodal vectors are read and written as (u_x, u_y) pairs of 16 bytes: the
// entry points reject caller pointers that are not 16-byte aligned.
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// An NVTX range around a public call (no cost without a profiler attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Shared by the translation units (defined in mto_api.cu).
mto_status enqueue_set_design(mto_ctx* c, int n_phase, const double* x_dev, const double* E_phase,
                              double penal);
mto_status enqueue_solve_core(mto_ctx* c);
mto_status enqueue_rhs_prologue(mto_ctx* c, const double* f_dev, const double* u_dev);
mto_status enqueue_rhs_epilogue(mto_ctx* c, double* u_dev, int rhs_slot);
mto_status enqueue_compliance(mto_ctx* c, int n_rhs, const double* f_dev, const double* u_dev,
                              double* compliance_dev, double* dcdx_dev);
void invalidate_graphs(mto_ctx* c);
// Makes `want` workspaces usable for concurrent right-hand sides (the context
// and want - 1 extra ones, created on first use, design state and launch
// shapes copied from c); *got is how many are usable (fewer if memory runs
// out).  Allocates: call outside any stream capture.
mto_status ensure_slots(mto_ctx* c, int want, int* got);
int target_warps(const mto_ctx* c, int level);
int target_warps64(const mto_ctx* c);

}  // namespace mto
