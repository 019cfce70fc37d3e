// dec_noalloc.cu - the boundary-flux sums of dec_k_eff as one entry point
// that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: code that runs inside a
// framework which owns every device allocation through its own pool, under
// a fixed device-memory budget, or where a device allocation would
// synchronise the device at the wrong moment.  They already hold the mesh
// arrays and the temperature field in memory of their own, so this entry
// point takes plain pointers and keeps its only scratch data (per-block
// partial sums and an arrival counter) in a fixed-size array that lives in
// the library's device image: every GPU that loads the library holds it
// until the process exits.
#include "dec_internal.cuh"

#include <mutex>

namespace dec {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 8;                                   // edges per thread
constexpr int kNaMaxBlocks = 32768;
constexpr int64_t kNaMaxEdges = (int64_t)kNaMaxBlocks * kNaThreads * kNaItems;

// [3 * kNaMaxBlocks] partial sums, then the arrival counter (as unsigned)
static __device__ __align__(256) double g_noalloc_scratch[3 * kNaMaxBlocks + 32];

__global__ void __launch_bounds__(kNaThreads)
k_eff_edges_kernel(const int32_t* __restrict__ E, int64_t ne, const double* __restrict__ w,
                   const double* __restrict__ T, const double* __restrict__ xyz,
                   const uint8_t* __restrict__ tag, double* scratch, double* out3) {
  double qin = 0.0, qout = 0.0, en = 0.0;
  const int64_t base = (int64_t)blockIdx.x * kNaThreads * kNaItems + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kNaItems; ++u) {
    const int64_t e = base + (int64_t)u * kNaThreads;
    if (e >= ne) break;
    const int32_t i = E[2 * e], j = E[2 * e + 1];
    const double d = T[i] - T[j];
    const double f = w[e] * d;          // heat flowing from i to j
    en += f * d;
    if (tag[i] == DEC_NODE_DIRICHLET) {
      const double xi = xyz[3 * (int64_t)i];
      if (xi == 0.0) qin += f; else if (xi == 1.0) qout -= f;
    }
    if (tag[j] == DEC_NODE_DIRICHLET) {
      const double xj = xyz[3 * (int64_t)j];
      if (xj == 0.0) qin -= f; else if (xj == 1.0) qout += f;
    }
  }
  double v[3] = {qin, qout, en}, t[3];
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + 3 * kNaMaxBlocks);
  if (grid_reduce<kNaThreads, 3>(v, t, scratch, ticket) && threadIdx.x == 0) {
    out3[0] = t[0];
    out3[1] = t[1];
    out3[2] = t[2];
  }
}

namespace {
std::mutex g_na_mutex;
double* g_na_ptr[64] = {nullptr};   // device address of the scratch array, per device
}  // namespace

}  // namespace dec

extern "C" dec_status dec_k_eff_edges_noalloc(int device, void* stream,
                                              const int32_t* E, int64_t n_edges,
                                              const double* w, const double* T,
                                              const double* xyz, const uint8_t* node_tag,
                                              double* out3) {
  using namespace dec;
  if (!E || !w || !T || !xyz || !node_tag || !out3 || n_edges < 1) return DEC_ERR_ARG;
  if (n_edges > kNaMaxEdges) return DEC_ERR_LIMIT;
  int n_devices = 0;
  if (cudaGetDeviceCount(&n_devices) != cudaSuccess) return DEC_ERR_CUDA;
  if (device < 0 || device >= 64 || device >= n_devices) return DEC_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return DEC_ERR_CUDA;
  double* scratch = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name
    // of the array is not its device address
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[device]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DEC_ERR_CUDA;
      g_na_ptr[device] = static_cast<double*>(p);
    }
    scratch = g_na_ptr[device];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + 3 * kNaMaxBlocks);
  // the arrival counter must start at zero (the last block also resets it)
  if (cudaMemsetAsync(ticket, 0, sizeof(unsigned), s) != cudaSuccess) return DEC_ERR_CUDA;
  const int64_t per_block = (int64_t)kNaThreads * kNaItems;
  const unsigned blocks = (unsigned)((n_edges + per_block - 1) / per_block);
  // the totals land in the tail of the scratch array, then go to out3
  double* res = scratch + 3 * kNaMaxBlocks + 8;
  k_eff_edges_kernel<<<blocks, kNaThreads, 0, s>>>(E, n_edges, w, T, xyz, node_tag, scratch,
                                                   res);
  if (cudaGetLastError() != cudaSuccess) return DEC_ERR_CUDA;
  if (cudaMemcpyAsync(out3, res, 3 * sizeof(double), cudaMemcpyDefault, s) != cudaSuccess)
    return DEC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DEC_ERR_CUDA;
  return DEC_OK;
}
