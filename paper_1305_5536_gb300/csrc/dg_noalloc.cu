// dg_noalloc.cu -- conservation totals of a caller-owned device state without
// any device allocation (dg_totals_noalloc in include/dg.h).
//
// Who needs it: callers that may not call cudaMalloc.  A simulation that has
// reserved nearly all of the GPU's memory for its own state cannot risk an
// allocation failing in the middle of a run; a framework that owns the device
// memory through its own pool forbids raw allocations; and code enqueuing work
// asynchronously cannot afford cudaMalloc/cudaFree, which may synchronise the
// device.  Such callers still want the FP64 compensated totals of the conserved
// variables (mass, momentum, energy, magnetic flux) of a state they hold.
//
// The per-block partial sums live in one file-scope __device__ array of fixed
// size, shared by every call on that device and kept until the process exits.
// Calls that overlap on the GPU race on it; enqueue them one after another.
#include <cuda_runtime.h>

#include <string>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr long kCellsPerBlock = (long)kThreads * kCellsPerThread;  // 4096
constexpr int kMaxBlocks = 4096;  // => at most 16,777,216 cells
constexpr int kMaxVars = 8;
// layout: [kMaxVars][kMaxBlocks][2] partial (sum, compensation) pairs, then
// kMaxVars results, then one slot whose first 4 bytes are the block ticket
constexpr int kResults = kMaxVars * kMaxBlocks * 2;
constexpr int kTicket = kResults + kMaxVars;
constexpr int kScratchDoubles = kTicket + 1;

// 32 KB x 8 = 512 KiB + 72 B of device memory per GPU that loads the library.
static __device__ __align__(256) double g_totals_scratch[kScratchDoubles];

struct Planes {
  int nv;
  int plane[kMaxVars];
};

__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

// One launch: every block sums its 4096 cells of every variable with Neumaier
// compensation; the last block to finish combines the partials in block order
// (deterministic) and writes the results.
__global__ void __launch_bounds__(kThreads) totals_static_kernel(const double* __restrict__ u,
                                                                 long ncell, Planes P,
                                                                 double* scratch, double vol) {
  __shared__ double ss[kThreads], cc[kThreads];
  __shared__ bool last;
  const long base = blockIdx.x * kCellsPerBlock;
  for (int v = 0; v < P.nv; ++v) {
    const double* plane = u + (size_t)P.plane[v] * ncell;
    double s = 0.0, c = 0.0;
    for (int k = 0; k < kCellsPerThread; ++k) {
      long i = base + (long)k * kThreads + threadIdx.x;
      if (i < ncell) neumaier(s, c, plane[i]);
    }
    ss[threadIdx.x] = s;
    cc[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      double S = 0.0, C = 0.0;
      for (int t = 0; t < kThreads; ++t) {
        neumaier(S, C, ss[t]);
        C += cc[t];
      }
      scratch[((size_t)v * kMaxBlocks + blockIdx.x) * 2] = S;
      scratch[((size_t)v * kMaxBlocks + blockIdx.x) * 2 + 1] = C;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kTicket);
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x < P.nv) {
    __threadfence();
    const int v = threadIdx.x;
    double S = 0.0, C = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      neumaier(S, C, scratch[((size_t)v * kMaxBlocks + b) * 2]);
      C += scratch[((size_t)v * kMaxBlocks + b) * 2 + 1];
    }
    scratch[kResults + v] = (S + C) * vol;
  }
  if (last && threadIdx.x == 0) *reinterpret_cast<unsigned int*>(scratch + kTicket) = 0u;
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// failures are reported through dg_last_error(NULL)
dg_status fail(dg_status s, const std::string& m) {
  dgk::set_global_error(m);
  return s;
}

}  // namespace

extern "C" dg_status dg_totals_noalloc(const dg_config* cfg, const double* u, double* out,
                                       int out_on_device, void* cuda_stream) {
  if (!cfg || !u || !out) return fail(DG_EINVAL, "null argument");
  if (cfg->eq != DG_EULER && cfg->eq != DG_MHD) return fail(DG_EINVAL, "eq must be DG_EULER or DG_MHD");
  if (cfg->dim != 2 && cfg->dim != 3) return fail(DG_EINVAL, "dim must be 2 or 3");
  long ncell = 1;
  for (int a = 0; a < cfg->dim; ++a) {
    if (cfg->n[a] < 1) return fail(DG_EINVAL, "grid size must be >= 1");
    if (!(cfg->box[a] > 0.0)) return fail(DG_EINVAL, "box lengths must be positive");
    ncell *= cfg->n[a];
  }
  const long blocks = (ncell + kCellsPerBlock - 1) / kCellsPerBlock;
  if (blocks > kMaxBlocks)
    return fail(DG_EINVAL,
                "grid too large for dg_totals_noalloc: at most 16777216 cells (4096 blocks of "
                "4096 cells) fit its static scratch; use dg_totals");
  // planes of the averages in the interchange layout
  Planes P;
  const int K = cfg->dim + 1;
  const int nT = cfg->dim == 2 ? 4 : 5;
  P.nv = 0;
  for (int v = 0; v < nT; ++v) P.plane[P.nv++] = v * K;
  if (cfg->eq == DG_MHD) {
    P.plane[P.nv++] = nT * K;
    P.plane[P.nv++] = nT * K + 1;
    if (cfg->dim == 3) P.plane[P.nv++] = nT * K + 2;
  }
  double vol = 1.0;
  for (int a = 0; a < cfg->dim; ++a) vol *= cfg->box[a] / cfg->n[a];

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(DG_ECUDA, "no usable CUDA device");
  }
  // Set-up on the first call on this device (with it current): the device
  // address of the scratch array.  Make this first call before any stream
  // capture.
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_totals_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(DG_ECUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  double* scratch = g_scratch_ptr[dev];
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the block ticket must start at zero
  if (cudaMemsetAsync(scratch + kTicket, 0, sizeof(double), st) != cudaSuccess) {
    cudaGetLastError();
    return fail(DG_ECUDA, "clearing the ticket failed");
  }
  totals_static_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(u, ncell, P, scratch, vol);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DG_ECUDA, cudaGetErrorString(e));
  e = cudaMemcpyAsync(out, scratch + kResults, P.nv * sizeof(double),
                      out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return fail(DG_ECUDA, cudaGetErrorString(e));
  if (!out_on_device) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(DG_ECUDA, cudaGetErrorString(e));
  }
  return DG_OK;
}
