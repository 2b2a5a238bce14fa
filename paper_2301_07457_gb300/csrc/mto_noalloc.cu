// Compliance and sensitivities without any device allocation.
//
// For callers that cannot allocate device memory: hosts whose memory pool
// owns all of HBM and forbids other allocations, and latency-critical loops that cannot afford the device-wide
// synchronisation of cudaMalloc/cudaFree.  The context-based
// mto_compliance_grad needs a context (allocated by mto_create_mesh); this
// entry point needs none.  Its reduction scratch (one partial per block plus
// the last-block ticket) is a fixed file-scope device array that every GPU
// loading the library holds until the process exits.
#include <mutex>

#include "mto_ctx.cuh"

using namespace mto;

namespace {

constexpr int NA_NT = 256;
constexpr int NA_NODES_PER_BLOCK = 4 * NA_NT;
constexpr int NA_MAX_BLOCKS = 32768;  // => at most 33,554,432 nodes
constexpr long long NA_MAX_NODES = (long long)NA_MAX_BLOCKS * NA_NODES_PER_BLOCK;
// Two partial sums per block (the shared reduction writes pairs), then the
// ticket in the last slot.  512 KiB.
constexpr int NA_SCRATCH_DOUBLES = 2 * NA_MAX_BLOCKS + 32;

static __device__ __align__(256) double g_noalloc_scratch[NA_SCRATCH_DOUBLES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mutex;
double* g_scratch_ptr[NA_MAX_DEVICES] = {};

// f . u over the dense node-interleaved layout: block b sums nodes
// [b * NA_NODES_PER_BLOCK, (b+1) * NA_NODES_PER_BLOCK), then the last block
// adds the block partials in order (deterministic, no floating-point atomics).
__global__ void __launch_bounds__(NA_NT)
    dot_noalloc_kernel(long long nodes, const double2* __restrict__ f, const double2* __restrict__ u,
                       double* scratch, double* out) {
  double acc = 0.0;
  const long long base = (long long)blockIdx.x * NA_NODES_PER_BLOCK;
  for (int t = threadIdx.x; t < NA_NODES_PER_BLOCK; t += NA_NT) {
    const long long k = base + t;
    if (k < nodes) {
      const double2 a = f[k], b = u[k];
      acc += a.x * b.x + a.y * b.y;
    }
  }
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + 2 * NA_MAX_BLOCKS);
  block_reduce_finish<NA_NT>(acc, 0.0, scratch, ticket, nullptr, FIN_NONE, out);
}

// The device address of the scratch array on `device`, looked up once per
// device with that device current.
cudaError_t scratch_for(int device, double** out) {
  if (device < 0 || device >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[device]) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" mto_status mto_compliance_grad_noalloc(int nelx, int nely, double nu, int n_phase,
                                                  const double* x_dev, const double* E_phase,
                                                  double penal, const double* f_dev,
                                                  const double* u_dev, double* compliance_dev,
                                                  double* dcdx_dev, int device, void* cuda_stream) {
  if (nelx < 1 || nely < 1 || !(nu > -1.0 && nu < 0.5) || n_phase < 1 || n_phase > 16 || !E_phase ||
      !(penal >= 1.0 && penal <= 64.0) || !f_dev || !u_dev || !compliance_dev || !aligned16(f_dev) ||
      !aligned16(u_dev) ||
      (dcdx_dev && !x_dev))
    return MTO_ERR_ARG;
  const long long nodes = ((long long)nelx + 1) * ((long long)nely + 1);
  if (nodes > NA_MAX_NODES) return MTO_ERR_UNSUPPORTED_MESH;
  for (int i = 0; i < n_phase; ++i)
    if (!(E_phase[i] > 0.0 && E_phase[i] < 1e300)) return MTO_ERR_ARG;
  // Every MTO_ERR_CUDA below records its cause for mto_cuda_error_string.
  auto fail = [](cudaError_t e) {
    g_last_cuda = e;
    return MTO_ERR_CUDA;
  };
  double* scratch = nullptr;
  cudaError_t e = scratch_for(device, &scratch);
  if (e != cudaSuccess) return fail(e);
  int prev = 0;
  e = cudaGetDevice(&prev);
  if (e == cudaSuccess) e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(e);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  mto_status st = MTO_OK;
  // The ticket must start at zero; the partials are always written before use.
  e = cudaMemsetAsync(scratch + 2 * NA_MAX_BLOCKS, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) {
    st = fail(e);
  } else {
    const int blocks = (int)((nodes + NA_NODES_PER_BLOCK - 1) / NA_NODES_PER_BLOCK);
    dot_noalloc_kernel<<<blocks, NA_NT, 0, s>>>(nodes, reinterpret_cast<const double2*>(f_dev),
                                                reinterpret_cast<const double2*>(u_dev), scratch,
                                                compliance_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = fail(e);
  }
  if (st == MTO_OK && dcdx_dev) {
    PhaseTable ph{};
    for (int i = 0; i < n_phase; ++i) ph.E[i] = E_phase[i];
    const int ipenal = (penal == (double)(int)penal && penal <= 16.0) ? (int)penal : -1;
    const double kap = 1.0 / (4.0 * (1.0 - nu * nu)), gs = 0.5 * (1.0 - nu);
    const FineConst<double> kf = {kap, kap * nu, kap * (1.0 + gs) / 3.0, kap * gs};
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    e = launch_sensitivity(nelx, nely, n_phase, x_dev, ph, penal, ipenal, kf, u_dev, dcdx_dev, 0, s, sms);
    if (e != cudaSuccess) st = fail(e);
  }
  cudaSetDevice(prev);
  return st;
}
