// dg_common.cuh -- shared device/host definitions of the DG kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_physics.cuh"

namespace dgk {

// Per-problem control block in device memory.  The Courant time step of the
// current state is cfl / vmax_cur; stage 2 of a step accumulates the signal speed
// of the new state into vmax_next (bit pattern of a positive double, so that the
// integer atomicMax orders it), and the last CTA to finish moves it to vmax_cur.
struct Ctl {
  double vmax_cur;
  double dt_cur;  // cfl / vmax_cur, formed once per step by whoever sets vmax_cur
  unsigned long long vmax_next;
  double t;
  double dt_last;
  long long step;
  unsigned int ticket;
  unsigned int err;
  double* dt_hist;      // optional record of the time steps (adjoint)
  long long hist_cap;
  long long err_step;   // step in which `err` was first raised (-1: never)
};

// One state: FP64 cell averages [nv][ncell] and derivative coefficients
// [ns][ncell] of type TS (double or float).
template <class TS>
struct StateBuf {
  double* c0;
  TS* sl;
};

// Constants of the equation of state in both arithmetic types, derived once on
// the host (deriving them per thread would put double divisions on the FP64 pipe).
struct GasPair {
  Gas<double> d;
  Gas<float> f;
  __host__ void set(double gamma) {
    d.set(gamma);
    f.set(gamma);
  }
};
template <class T> __device__ __forceinline__ const Gas<T>& gas_of(const GasPair& g);
template <> __device__ __forceinline__ const Gas<double>& gas_of<double>(const GasPair& g) { return g.d; }
template <> __device__ __forceinline__ const Gas<float>& gas_of<float>(const GasPair& g) { return g.f; }

// Phase profiling of the stage kernels, compiled in only by the profiling build
// (-DDG_PHASE_PROFILE; the normal build has no stamps).  Thread 0 of every CTA
// stamps clock64() at the end of each phase -- after the barrier that closes it,
// or after its own work where no barrier follows -- and adds the SM cycles since
// its previous stamp to that phase's counter: acc[(stage - 1) * kPhaseSlots +
// phase].  Summed over the CTAs, the counters give each phase's share of the
// kernel's time.
constexpr int kPhaseSlots = 16;
struct PhaseStamp {
#ifdef DG_PHASE_PROFILE
  long long t;
  unsigned long long* acc;
  __device__ __forceinline__ void begin(unsigned long long* a, int stage) {
    acc = a ? a + (stage - 1) * kPhaseSlots : nullptr;
    t = clock64();
  }
  __device__ __forceinline__ void mark(int phase) {
    if (acc && threadIdx.x == 0) {
      const long long now = clock64();
      atomicAdd(acc + phase, (unsigned long long)(now - t));
      t = now;
    }
  }
#else
  __device__ __forceinline__ void begin(unsigned long long*, int) {}
  __device__ __forceinline__ void mark(int) {}
#endif
};

// Arguments of one stage launch on one periodic 2D grid.
template <class TS>
struct Stage2DArgs {
  int nx, ny;
  long ncell;
  double dx, dy;
  double gamma, cfl, dt_override;
  GasPair gas;
  int limiter;
  StateBuf<TS> in;    // stage input (V^n in stage 1, V^1 in stage 2)
  StateBuf<TS> base;  // V^n (stage 2 only)
  StateBuf<TS> out;
  // Limited derivative coefficients of U^n = Lambda(V^n): stage 1 stores those of
  // its own cells here (the step's output buffer), stage 2 reads them back for its
  // own cell before overwriting it.  Null: stage 2 recomputes them.
  TS* lim_sl;
  Ctl* ctl;
  // Largest grid of a persistent launch (the TMA kernels), 0 = as many CTAs as are
  // resident.  Set only by a test hook, so that each CTA walks many tiles.
  int max_ctas = 0;
  unsigned long long* phase = nullptr;  // phase cycle counters (profiling build)
};

// Arguments of one stage launch on one periodic 3D grid.
template <class TS>
struct Stage3DArgs {
  int nx, ny, nz;
  long ncell;
  double dx, dy, dz;
  double gamma, cfl, dt_override;
  GasPair gas;
  int limiter;
  StateBuf<TS> in;
  StateBuf<TS> base;
  StateBuf<TS> out;
  TS* lim_sl;  // as for Stage2DArgs
  Ctl* ctl;
  unsigned long long* phase = nullptr;  // phase cycle counters (profiling build)
};

// The cells of a TX x TY x TZ tile and its six face slabs (the halo-1 box
// without its edges and corners): the cells whose limited slopes the face fluxes
// read.  Cell e (0 <= e < ring3d_count) as halo-1 box coordinates (rx, ry, rz):
// first the tile, then the x, y and z slabs (low side, then high side).
template <int TX, int TY, int TZ>
__host__ __device__ constexpr int ring3d_count() {
  return TX * TY * TZ + 2 * (TY * TZ + TX * TZ + TX * TY);
}
template <int TX, int TY, int TZ>
__host__ __device__ __forceinline__ void ring3d_cell(int e, int& rx, int& ry, int& rz) {
  constexpr int NT = TX * TY * TZ, SX = TY * TZ, SY = TX * TZ, SZ = TX * TY;
  if (e < NT) {
    rx = e % TX + 1; ry = (e / TX) % TY + 1; rz = e / (TX * TY) + 1;
  } else if (e < NT + 2 * SX) {
    const int k = e - NT, s = k >= SX, q = k - s * SX;
    rx = s ? TX + 1 : 0; ry = q % TY + 1; rz = q / TY + 1;
  } else if (e < NT + 2 * (SX + SY)) {
    const int k = e - NT - 2 * SX, s = k >= SY, q = k - s * SY;
    ry = s ? TY + 1 : 0; rx = q % TX + 1; rz = q / TX + 1;
  } else {
    const int k = e - NT - 2 * (SX + SY), s = k >= SZ, q = k - s * SZ;
    rz = s ? TZ + 1 : 0; rx = q % TX + 1; ry = q / TX + 1;
  }
}

// The cells of the halo-2 box whose centroid primitives the limiter of the tile
// and its face slabs reads: the halo-1 box and, beyond each face of the tile, one
// more layer of the tile's extent (the outer neighbours of the slabs).  Cell e
// (0 <= e < halo3d_count) as halo-2 box coordinates (rx, ry, rz): first the halo-1
// box in its own row-major order (so e is the cell's halo-1 index), then the x, y
// and z layers (low side, then high side).
template <int TX, int TY, int TZ>
__host__ __device__ constexpr int halo3d_count() {
  return (TX + 2) * (TY + 2) * (TZ + 2) + 2 * (TY * TZ + TX * TZ + TX * TY);
}
template <int TX, int TY, int TZ>
__host__ __device__ __forceinline__ void halo3d_cell(int e, int& rx, int& ry, int& rz) {
  constexpr int R1X = TX + 2, R1Y = TY + 2, R1 = R1X * R1Y * (TZ + 2);
  constexpr int SX = TY * TZ, SY = TX * TZ, SZ = TX * TY;
  if (e < R1) {
    rz = e / (R1X * R1Y);
    const int q = e - rz * (R1X * R1Y);
    ry = q / R1X;
    rx = q - ry * R1X + 1;
    ry += 1;
    rz += 1;
  } else if (e < R1 + 2 * SX) {
    const int k = e - R1, s = k >= SX, q = k - s * SX;
    rx = s ? TX + 3 : 0; ry = q % TY + 2; rz = q / TY + 2;
  } else if (e < R1 + 2 * (SX + SY)) {
    const int k = e - R1 - 2 * SX, s = k >= SY, q = k - s * SY;
    ry = s ? TY + 3 : 0; rx = q % TX + 2; rz = q / TX + 2;
  } else {
    const int k = e - R1 - 2 * (SX + SY), s = k >= SZ, q = k - s * SZ;
    rz = s ? TZ + 3 : 0; rx = q % TX + 2; ry = q / TX + 2;
  }
}

// Division of small non-negative integers by a divisor known only at run time (a
// face count of a rolled loop over orientations): floor(n / d) = (n * m) >> 32
// with m = ceil(2^32 / d), exact for n < 2^14 and 2 <= d <= 1024 (checked for
// every such pair; d = 1 would need m = 2^32); two instructions instead of a full
// integer division.
__host__ __device__ __forceinline__ unsigned div_magic(unsigned d) {
  return (unsigned)((0x100000000ull + d - 1) / d);
}
__host__ __device__ __forceinline__ int div_by_magic(int n, unsigned m) {
#ifdef __CUDA_ARCH__
  return (int)__umulhi((unsigned)n, m);
#else
  return (int)(((unsigned long long)(unsigned)n * m) >> 32);
#endif
}

__host__ __device__ __forceinline__ int wrap_index(int g, int n) {
  int r = g % n;
  return r < 0 ? r + n : r;
}

// Programmatic dependent launch: a kernel launched with the programmatic stream-
// serialisation attribute may be scheduled while the kernel before it on the stream
// is finishing.  griddep_wait() returns once that kernel has completed and its
// writes are visible (at once for a normal launch); griddep_launch_dependents() lets
// the launch of the next kernel on the stream begin.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Launch of a stage kernel as a programmatic dependent of the kernel before it on
// the stream (the kernel must begin with griddep_wait()).
template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Global -> shared copy of one 4- or 8-byte element without a register round
// trip (cp.async); cp_async_wait_all() waits for this thread's copies.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8, "element copies of 4 or 8 bytes");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Request the line holding `p` into L2 (no register, no wait): for global reads
// that come later in a kernel, so that they find the line in L2.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

}  // namespace dgk
