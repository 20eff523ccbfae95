// dg_capi.cu -- host side of the C ABI declared in include/dg.h: contexts,
// device memory, layout conversion, stepping (direct launches or CUDA-graph
// replay), diagnostics, kernel timing and the tile-shape autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dg.h"
#include "dg_adjoint.h"
#include "dg_batch.h"
#include "dg_internal.h"

using namespace dgk;

namespace {

struct Prob {
  dg_config cfg;
  int nx, ny, nz;
  long ncell;
  double dx, dy, dz;
  size_t c0_off, sl_off;  // element offsets of this problem inside the state arrays
  size_t plane_off;       // offset in the concatenated interchange array
};

struct EvPair {
  cudaEvent_t a, b;
  int kind;
};

}  // namespace

struct dg_ctx {
  std::vector<Prob> probs;
  int eq = 0, dim = 2, fp32 = 0, limiter = 1, ckpt_every = 0;
  int integrator = DG_SSPRK2, face_points = 2;  // face rule of the MUSCL-Hancock step
  double gamma = 1.4, cfl = 0.3;
  int nplanes = 0, nv = 0, ns = 0;
  PlaneMap pmap{};
  long ncell_total = 0;
  cudaStream_t stream = nullptr;      // caller's stream: every launch and copy
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  cudaStream_t launch_stream = nullptr;
  // three state buffers: current (cur), stage-1 output (1), next
  double* c0[3] = {nullptr, nullptr, nullptr};
  void* sl[3] = {nullptr, nullptr, nullptr};
  int cur = 0, nxt = 2;
  Ctl* ctl = nullptr;       // device, one per problem
  Ctl* ctl_host = nullptr;  // pinned mirror for readback
  double* scratch = nullptr;  // device, one interchange plane (host transfers, totals)
  size_t scratch_elems = 0;
  double* totals_dev = nullptr;
  int variant = -1;  // tile shape (-1: not tuned yet)
  bool state_set = false;
  std::string err;
  // CUDA graphs of two steps, keyed by (cur buffer, dt_override)
  std::map<std::pair<int, double>, cudaGraphExec_t> graphs;
  // kernel timing
  bool prof = false;
  std::vector<EvPair> evs;
  // adjoint recording
  AdjointStore adj;
  // batched 2D problems: one persistent launch per step over a tile work list
  bool batch2d = false;
  BatchProb* btab[3] = {nullptr, nullptr, nullptr};  // per tile variant of the batch kernel
  int btiles[3] = {0, 0, 0};
  unsigned* bar = nullptr;
  long long spin_limit = 1LL << 24;
  int extra_arrivals = 0;
  // test hook DG_TEST_MAX_CTAS: cap on the grids of the persistent (TMA, batched)
  // kernels, so that every CTA processes many tiles
  int max_ctas = 0;
  // phase cycle counters of the stage kernels (profiling build; 2 stages x
  // kPhaseSlots), allocated and cleared when profiling is enabled
  unsigned long long* phase_dev = nullptr;
  std::string kname;
};

namespace {

thread_local std::string g_err;

dg_status fail(dg_ctx* c, dg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_err = buf;
  return s;
}

#define CK(c, call)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail((c), DG_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                     \
  } while (0)

int nplanes_of(int eq, int dim) {
  int nT = (dim == 2) ? 4 : 5;
  return nT * (dim + 1) + (eq == DG_MHD ? (dim == 2 ? 5 : 11) : 0);
}

const char* validate(const dg_config* c) {
  if (!c) return "null configuration";
  if (c->eq != DG_EULER && c->eq != DG_MHD) return "eq must be DG_EULER or DG_MHD";
  if (c->dim != 2 && c->dim != 3) return "dim must be 2 or 3";
  for (int a = 0; a < c->dim; ++a) {
    if (c->n[a] < 1 || c->n[a] > (1 << 20)) return "grid size out of range";
    if (!(c->box[a] > 0.0) || !std::isfinite(c->box[a])) return "box lengths must be positive";
  }
  double cells = (double)c->n[0] * c->n[1] * (c->dim == 3 ? c->n[2] : 1);
  if (cells > 2.0e9) return "too many cells";
  if (!(c->gamma > 1.0) || !std::isfinite(c->gamma)) return "gamma must be > 1";
  if (!(c->cfl > 0.0) || !std::isfinite(c->cfl)) return "cfl must be > 0";
  if (c->limiter < 0 || c->limiter > 2)
    return "limiter must be 0 (off), 1 (min/max) or 2 (WENO-type)";
  if (c->precision != DG_FP64 && c->precision != DG_FP32) return "precision must be DG_FP64 or DG_FP32";
  if (c->eq == DG_EULER && c->riemann != DG_EXACT) return "Euler uses the exact Riemann solver (DG_EXACT)";
  if (c->eq == DG_MHD && c->riemann != DG_HLLD) return "MHD uses the HLLD solver (DG_HLLD)";
  if (c->ckpt_every < 0) return "ckpt_every must be >= 0";
  if (c->integrator != DG_SSPRK2 && c->integrator != DG_MUSCL_HANCOCK)
    return "integrator must be DG_SSPRK2 or DG_MUSCL_HANCOCK";
  if (c->face_points < 0 || c->face_points > 2) return "face_points must be 0, 1 or 2";
  if (c->integrator == DG_SSPRK2 && c->face_points == 1)
    return "the SSP-RK2 step uses the Gauss face rule (face_points 0 or 2)";
  return nullptr;
}

void build_plane_map(dg_ctx* c) {
  // Taylor variable v, coefficient k: average v (k = 0) or slope v*dim + (k-1)
  int nT = c->dim == 2 ? 4 : 5;
  PlaneMap& m = c->pmap;
  m.nplanes = c->nplanes;
  int p = 0;
  for (int v = 0; v < nT; ++v)
    for (int k = 0; k <= c->dim; ++k, ++p) {
      m.kind[p] = k == 0 ? 0 : 1;
      m.idx[p] = k == 0 ? v : v * c->dim + (k - 1);
    }
  if (c->eq == DG_MHD && c->dim == 2) {  // b1, b2 averages 4, 5; a1, a2, a3 slopes 8, 9, 10
    m.kind[p] = 0; m.idx[p++] = 4;
    m.kind[p] = 0; m.idx[p++] = 5;
    m.kind[p] = 1; m.idx[p++] = 8;
    m.kind[p] = 1; m.idx[p++] = 9;
    m.kind[p] = 1; m.idx[p++] = 10;
  } else if (c->eq == DG_MHD) {  // b1..b3 averages 5..7; a4..a11 slopes 15..22
    for (int k = 0; k < 3; ++k) { m.kind[p] = 0; m.idx[p++] = 5 + k; }
    for (int k = 0; k < 8; ++k) { m.kind[p] = 1; m.idx[p++] = 15 + k; }
  }
  c->nv = nT + (c->eq == DG_MHD ? c->dim : 0);
  c->ns = nT * c->dim + (c->eq == DG_MHD ? (c->dim == 2 ? 3 : 8) : 0);
}

template <class TS>
StateBuf<TS> sbuf(dg_ctx* c, int b, const Prob& p) {
  StateBuf<TS> s;
  s.c0 = c->c0[b] + p.c0_off;
  s.sl = reinterpret_cast<TS*>(c->sl[b]) + p.sl_off;
  return s;
}

dg_status alloc_ctx(dg_ctx* c) {
  size_t c0n = 0, sln = 0;
  for (auto& p : c->probs) {
    p.c0_off = c0n;
    p.sl_off = sln;
    c0n += (size_t)c->nv * p.ncell;
    sln += (size_t)c->ns * p.ncell;
  }
  size_t ts = c->fp32 ? sizeof(float) : sizeof(double);
  for (int b = 0; b < 3; ++b) {
    if (cudaMalloc(&c->c0[b], c0n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->sl[b], sln * ts) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, DG_ENOMEM, "device allocation of the state failed (%.2f GB)",
                  3.0 * (c0n * 8.0 + sln * ts) / 1e9);
    }
  }
  long maxcell = 0;
  for (auto& p : c->probs) maxcell = std::max(maxcell, p.ncell);
  c->scratch_elems = std::max<size_t>((size_t)maxcell, 256 * 2 * 8);
  CK(c, cudaMalloc(&c->scratch, c->scratch_elems * sizeof(double)));
  CK(c, cudaMalloc(&c->ctl, c->probs.size() * sizeof(Ctl)));
  CK(c, cudaMemset(c->ctl, 0, c->probs.size() * sizeof(Ctl)));
  CK(c, cudaMallocHost(&c->ctl_host, c->probs.size() * sizeof(Ctl)));
  CK(c, cudaMalloc(&c->totals_dev, 16 * sizeof(double)));
  return DG_OK;
}

void free_graphs(dg_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

// ---------------------------------------------------------------------------
// stage launches
// ---------------------------------------------------------------------------
// Tile shapes compiled for the batched kernel (one work list each).
constexpr int kBatchVariants = 3;

template <class TS>
cudaError_t launch_batch_step_t(dg_ctx* c, int a, int b, double dtov) {
  const int v = c->variant < 0 ? 0 : c->variant;
  if (v >= kBatchVariants) return cudaErrorInvalidValue;  // no work list for it
  BatchArgs<TS> B;
  B.probs = c->btab[v];
  B.nprob = (int)c->probs.size();
  B.ntiles = c->btiles[v];
  B.gamma = c->gamma;
  B.gas.set(c->gamma);
  B.cfl = c->cfl;
  B.dt_override = dtov;
  B.limiter = c->limiter;
  const int bufs[3] = {a, 1, b};
  for (int k = 0; k < 3; ++k) {
    B.c0[k] = c->c0[bufs[k]];
    B.sl[k] = reinterpret_cast<TS*>(c->sl[bufs[k]]);
  }
  B.ctl = c->ctl;
  B.bar = c->bar;
  B.spin_limit = c->spin_limit;
  B.barrier_extra = c->extra_arrivals;
  B.max_ctas = c->max_ctas;
  return launch_batch2d(c->eq, v, B, c->launch_stream, nullptr);
}

template <class TS>
cudaError_t launch_stage_t(dg_ctx* c, int stage, int in, int base, int out, double dtov,
                           int lim) {
  for (size_t ip = 0; ip < c->probs.size(); ++ip) {
    const Prob& p = c->probs[ip];
    if (c->dim == 2) {
      Stage2DArgs<TS> a;
      a.nx = p.nx; a.ny = p.ny; a.ncell = p.ncell;
      a.dx = p.dx; a.dy = p.dy;
      a.gamma = c->gamma; a.cfl = c->cfl; a.dt_override = dtov; a.limiter = c->limiter;
      a.gas.set(c->gamma);
      a.in = sbuf<TS>(c, in, p);
      a.base = sbuf<TS>(c, base, p);
      a.out = sbuf<TS>(c, out, p);
      a.lim_sl = lim >= 0 ? sbuf<TS>(c, lim, p).sl : nullptr;
      a.ctl = c->ctl + ip;
      a.max_ctas = c->max_ctas;
      a.phase = c->prof ? c->phase_dev : nullptr;
      cudaError_t e = launch_stage2d(c->eq, c->variant < 0 ? 0 : c->variant, stage, a,
                                     c->launch_stream);
      if (e != cudaSuccess) return e;
    } else {
      Stage3DArgs<TS> a;
      a.nx = p.nx; a.ny = p.ny; a.nz = p.nz; a.ncell = p.ncell;
      a.dx = p.dx; a.dy = p.dy; a.dz = p.dz;
      a.gamma = c->gamma; a.cfl = c->cfl; a.dt_override = dtov; a.limiter = c->limiter;
      a.gas.set(c->gamma);
      a.in = sbuf<TS>(c, in, p);
      a.base = sbuf<TS>(c, base, p);
      a.out = sbuf<TS>(c, out, p);
      a.lim_sl = lim >= 0 ? sbuf<TS>(c, lim, p).sl : nullptr;
      a.ctl = c->ctl + ip;
      a.phase = c->prof ? c->phase_dev : nullptr;
      const int v = c->variant < 0 ? 0 : c->variant;
      cudaError_t e = c->eq == DG_MHD ? launch_stage3m(v, stage, a, c->launch_stream)
                                      : launch_stage3d(v, stage, a, c->launch_stream);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// `lim`: buffer receiving the limited derivative coefficients of the step input
// (the step's output buffer), or -1.
cudaError_t launch_stage(dg_ctx* c, int stage, int in, int base, int out, double dtov, int lim) {
  return c->fp32 ? launch_stage_t<float>(c, stage, in, base, out, dtov, lim)
                 : launch_stage_t<double>(c, stage, in, base, out, dtov, lim);
}

// One MUSCL-Hancock step of every problem from buffer `a` into buffer `b`.
template <class TS>
cudaError_t launch_mh_t(dg_ctx* c, int a, int b, double dtov) {
  const int v = c->variant < 0 ? 0 : c->variant;
  for (size_t ip = 0; ip < c->probs.size(); ++ip) {
    const Prob& p = c->probs[ip];
    if (c->dim == 3) {
      Stage3DArgs<TS> s;
      s.nx = p.nx; s.ny = p.ny; s.nz = p.nz; s.ncell = p.ncell;
      s.dx = p.dx; s.dy = p.dy; s.dz = p.dz;
      s.gamma = c->gamma; s.cfl = c->cfl; s.dt_override = dtov; s.limiter = c->limiter;
      s.gas.set(c->gamma);
      s.in = sbuf<TS>(c, a, p);
      s.base = s.in;
      s.out = sbuf<TS>(c, b, p);
      s.lim_sl = nullptr;
      s.ctl = c->ctl + ip;
      cudaError_t e = c->eq == DG_MHD ? launch_mh3m(v, c->face_points, s, c->launch_stream)
                                      : launch_mh3d(v, c->face_points, s, c->launch_stream);
      if (e != cudaSuccess) return e;
      continue;
    }
    Stage2DArgs<TS> s;
    s.nx = p.nx; s.ny = p.ny; s.ncell = p.ncell;
    s.dx = p.dx; s.dy = p.dy;
    s.gamma = c->gamma; s.cfl = c->cfl; s.dt_override = dtov; s.limiter = c->limiter;
    s.gas.set(c->gamma);
    s.in = sbuf<TS>(c, a, p);
    s.base = s.in;
    s.out = sbuf<TS>(c, b, p);
    s.lim_sl = nullptr;
    s.ctl = c->ctl + ip;
    cudaError_t e = launch_mh2d(c->eq, v, c->face_points, s, c->launch_stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One step from buffer `a` into buffer `b` (SSP-RK2: buffer 1 holds V^1).
cudaError_t launch_step(dg_ctx* c, int a, int b, double dtov) {
  if (c->integrator == DG_MUSCL_HANCOCK)
    return c->fp32 ? launch_mh_t<float>(c, a, b, dtov) : launch_mh_t<double>(c, a, b, dtov);
  if (c->batch2d)
    return c->fp32 ? launch_batch_step_t<float>(c, a, b, dtov) : launch_batch_step_t<double>(c, a, b, dtov);
  cudaError_t e = launch_stage(c, 1, a, a, 1, dtov, b);
  if (e != cudaSuccess) return e;
  return launch_stage(c, 2, 1, a, b, dtov, b);
}

cudaError_t launch_step_profiled(dg_ctx* c, int a, int b, double dtov) {
  if (c->batch2d || c->integrator == DG_MUSCL_HANCOCK) {
    EvPair ev;
    ev.kind = 1;
    cudaEventCreate(&ev.a);
    cudaEventCreate(&ev.b);
    cudaEventRecord(ev.a, c->stream);
    cudaError_t e = launch_step(c, a, b, dtov);
    cudaEventRecord(ev.b, c->stream);
    c->evs.push_back(ev);
    return e;
  }
  for (int s = 1; s <= 2; ++s) {
    EvPair ev;
    ev.kind = s - 1;
    cudaEventCreate(&ev.a);
    cudaEventCreate(&ev.b);
    cudaEventRecord(ev.a, c->stream);
    cudaError_t e = s == 1 ? launch_stage(c, 1, a, a, 1, dtov, b) : launch_stage(c, 2, 1, a, b, dtov, b);
    cudaEventRecord(ev.b, c->stream);
    c->evs.push_back(ev);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

dg_status ensure_graph(dg_ctx* c, double dtov, cudaGraphExec_t* out) {
  auto key = std::make_pair(c->cur, dtov);
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    *out = it->second;
    return DG_OK;
  }
  // capture on the private stream (the caller's may be the legacy default
  // stream, which cannot be captured); the graph is launched on the caller's
  cudaGraph_t g;
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  c->launch_stream = c->cap_stream;
  cudaError_t e1 = launch_step(c, c->cur, c->nxt, dtov);
  cudaError_t e2 = launch_step(c, c->nxt, c->cur, dtov);
  c->launch_stream = c->stream;
  cudaError_t e3 = cudaStreamEndCapture(c->cap_stream, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
    return fail(c, DG_ECUDA, "graph capture failed: %s",
                cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)));
  cudaGraphExec_t ex;
  cudaError_t e4 = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e4 != cudaSuccess) return fail(c, DG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e4));
  c->graphs[key] = ex;
  *out = ex;
  return DG_OK;
}

dg_status read_ctl(dg_ctx* c) {
  CK(c, cudaMemcpyAsync(c->ctl_host, c->ctl, c->probs.size() * sizeof(Ctl), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return DG_OK;
}

dg_status check_err(dg_ctx* c) {
  dg_status s = read_ctl(c);
  if (s != DG_OK) return s;
  for (size_t p = 0; p < c->probs.size(); ++p) {
    unsigned e = c->ctl_host[p].err;
    if (e & ERR_TIMEOUT) {
      // leave the context usable: clear the barrier and the error words (the
      // state of the failed step is unreliable; set it again to continue)
      CK(c, cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), c->stream));
      for (size_t q = 0; q < c->probs.size(); ++q)
        CK(c, cudaMemsetAsync((char*)(c->ctl + q) + offsetof(Ctl, err), 0, sizeof(unsigned),
                              c->stream));
      CK(c, cudaStreamSynchronize(c->stream));
      return fail(c, DG_ETIMEOUT, "grid barrier of the batched step timed out (step %lld)",
                  (long long)c->ctl_host[p].step);
    }
    if (e)
      return fail(c, DG_ENONPHYS,
                  "problem %zu: device error word 0x%x (1 non-physical state, 2 Riemann vacuum, "
                  "4 Newton iteration did not converge), first raised in step %lld (now after "
                  "step %lld)",
                  p, e, (long long)c->ctl_host[p].err_step, (long long)c->ctl_host[p].step);
  }
  return DG_OK;
}

// Initial Courant speed of the current state of every problem.
template <class TS>
dg_status init_cfl_t(dg_ctx* c) {
  for (size_t ip = 0; ip < c->probs.size(); ++ip) {
    const Prob& p = c->probs[ip];
    CK(c, launch_cfl<TS>(c->eq, c->dim, sbuf<TS>(c, c->cur, p), p.nx, p.ny, p.nz, p.dx, p.dy, p.dz,
                         c->gamma, c->ctl + ip, c->stream));
  }
  return DG_OK;
}

dg_status reset_ctl_and_cfl(dg_ctx* c) {
  CK(c, launch_ctl_reset(c->ctl, (int)c->probs.size(), c->stream));
  if (c->bar) CK(c, cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), c->stream));
  dg_status s = c->fp32 ? init_cfl_t<float>(c) : init_cfl_t<double>(c);
  if (s != DG_OK) return s;
  CK(c, launch_ctl_commit(c->ctl, (int)c->probs.size(), c->cfl, c->stream));
  return DG_OK;
}

// ---------------------------------------------------------------------------
// autotuner: time every compiled tile shape on the current state (scratch
// copies, the state is restored) and keep the fastest; cached per process by
// (eq, dim, precision, grid) and, if DG_TUNE_CACHE names a file, across runs.
// ---------------------------------------------------------------------------
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;
// contexts may be created and stepped from several host threads: one tuning at a
// time (this also keeps concurrent trial steps from timing each other)
std::mutex g_tune_mutex;

std::string tune_key(dg_ctx* c) {
  char b[128];
  const Prob& p = c->probs[0];
  snprintf(b, sizeof(b), "eq%d_d%d_fp%d_lim%d_%dx%dx%d_np%zu", c->eq, c->dim, c->fp32 ? 32 : 64,
           c->limiter, p.nx, p.ny, p.nz, c->probs.size());
  std::string k = b;
  if (c->integrator == DG_MUSCL_HANCOCK) k += "_mh" + std::to_string(c->face_points);
  return k;
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("DG_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[128];
  int v;
  while (fscanf(f, "%127s %d", key, &v) == 2) g_tune[key] = v;
  fclose(f);
}

void tune_save() {
  const char* path = getenv("DG_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "w");
  if (!f) return;
  for (auto& kv : g_tune) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
  fclose(f);
}

dg_status autotune(dg_ctx* c) {
  if (c->variant >= 0) return DG_OK;
  int nvar = c->integrator == DG_MUSCL_HANCOCK
                 ? (c->dim == 2 ? mh2d_variants(c->eq, c->fp32)
                    : (c->eq == DG_MHD ? mh3m_variants(c->fp32) : mh3d_variants(c->fp32)))
             : c->batch2d ? kBatchVariants
             : (c->dim == 2 ? stage2d_variants(c->eq, c->fp32)
                : (c->eq == DG_MHD ? stage3m_variants(c->fp32) : stage3d_variants(c->fp32)));
  // an explicit choice (DG_TILE_VARIANT) wins over the tuning cache when this
  // kind of context has that tile shape
  const char* env = getenv("DG_TILE_VARIANT");
  if (env) {
    const int v = atoi(env);
    if (v >= 0 && v < nvar) {
      c->variant = v;
      return DG_OK;
    }
  }
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load();
  std::string key = tune_key(c);
  auto it = g_tune.find(key);
  if (it != g_tune.end() && it->second >= 0 && it->second < nvar) {
    c->variant = it->second;
    return DG_OK;
  }
  if (nvar <= 1) {
    c->variant = 0;
    return DG_OK;
  }
  // time a fixed dt so that the trial steps do not depend on each other
  if (read_ctl(c) != DG_OK) return DG_ECUDA;
  double vmax = c->ctl_host[0].vmax_cur;
  double dt = vmax > 0.0 ? 0.25 * c->cfl / vmax : 1e-6;
  cudaEvent_t e0, e1;
  CK(c, cudaEventCreate(&e0));
  CK(c, cudaEventCreate(&e1));
  float best = 1e30f;
  int bestv = 0;
  Ctl saved[1];
  for (int v = 0; v < nvar; ++v) {
    c->variant = v;
    float tot = 0.0f;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {
      CK(c, cudaEventRecord(e0, c->stream));
      if (launch_step(c, c->cur, c->nxt, dt) != cudaSuccess) {
        // this shape does not apply to the grid (e.g. TMA rows not 16-byte aligned)
        cudaGetLastError();
        ok = false;
        break;
      }
      CK(c, cudaEventRecord(e1, c->stream));
      CK(c, cudaEventSynchronize(e1));
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tot += ms;
    }
    if (ok && tot < best) {
      best = tot;
      bestv = v;
    }
  }
  (void)saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->variant = bestv;
  g_tune[key] = bestv;
  tune_save();
  // the trial steps advanced the counters: restore them
  return reset_ctl_and_cfl(c);
}

// Device address of page-locked (pinned or registered) host memory, or null for
// pageable memory.  The layout kernels read and write such memory in place (over
// NVLink-C2C on Grace-Blackwell), so a state crosses the link once, without the
// per-plane staging copies through device scratch that pageable memory needs.
static void* mapped_view(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

template <class TS>
static dg_status set_state_t(dg_ctx* c, const double* src, int on_device) {
  if (!on_device) {
    if (const double* view = static_cast<const double*>(mapped_view(src))) {
      src = view;
      on_device = 1;
    }
  }
  for (const Prob& p : c->probs) {
    StateBuf<TS> dst = sbuf<TS>(c, c->cur, p);
    if (on_device) {
      CK(c, launch_state_in<TS>(src + p.plane_off, dst, c->pmap, p.ncell, c->stream));
      continue;
    }
    for (int k = 0; k < c->nplanes; ++k) {
      const double* plane = src + p.plane_off + (size_t)k * p.ncell;
      const double* dsrc = plane;
      if (!on_device) {
        CK(c, cudaMemcpyAsync(c->scratch, plane, p.ncell * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
        dsrc = c->scratch;
      }
      CK(c, launch_plane_in<TS>(dsrc, dst, c->pmap.kind[k], c->pmap.idx[k], p.ncell, c->stream));
    }
  }
  return DG_OK;
}

template <class TS>
static dg_status get_state_t(dg_ctx* c, double* dst, int on_device) {
  if (!on_device) {
    if (double* view = static_cast<double*>(mapped_view(dst))) {
      dst = view;
      on_device = 1;
    }
  }
  for (const Prob& p : c->probs) {
    StateBuf<TS> src = sbuf<TS>(c, c->cur, p);
    if (on_device) {
      CK(c, launch_state_out<TS>(src, dst + p.plane_off, c->pmap, p.ncell, c->stream));
      continue;
    }
    for (int k = 0; k < c->nplanes; ++k) {
      double* plane = dst + p.plane_off + (size_t)k * p.ncell;
      double* ddst = on_device ? plane : c->scratch;
      CK(c, launch_plane_out<TS>(src, ddst, c->pmap.kind[k], c->pmap.idx[k], p.ncell, c->stream));
      if (!on_device)
        CK(c, cudaMemcpyAsync(plane, c->scratch, p.ncell * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
    }
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return DG_OK;
}

}  // namespace

void dgk::set_global_error(const std::string& msg) { g_err = msg; }

namespace {

// Tile work lists of a 2D batch, one per compiled tile shape, and the barrier.
dg_status build_batch(dg_ctx* c) {
  c->batch2d = true;
  for (int v = 0; v < 3; ++v) {
    const int tx = batch2d_tile_x(c->fp32, v), ty = batch2d_tile_y(c->fp32, v);
    std::vector<BatchProb> tab;
    int begin = 0;
    for (const Prob& p : c->probs) {
      BatchProb b{};
      b.nx = p.nx;
      b.ny = p.ny;
      b.tiles_x = (p.nx + tx - 1) / tx;
      b.ntiles = b.tiles_x * ((p.ny + ty - 1) / ty);
      b.tile_begin = begin;
      b.ncell = p.ncell;
      b.dx = p.dx;
      b.dy = p.dy;
      b.c0_off = (long)p.c0_off;
      b.sl_off = (long)p.sl_off;
      begin += b.ntiles;
      tab.push_back(b);
    }
    c->btiles[v] = begin;
    CK(c, cudaMalloc(&c->btab[v], tab.size() * sizeof(BatchProb)));
    CK(c, cudaMemcpy(c->btab[v], tab.data(), tab.size() * sizeof(BatchProb), cudaMemcpyHostToDevice));
  }
  CK(c, cudaMalloc(&c->bar, 2 * sizeof(unsigned)));
  CK(c, cudaMemset(c->bar, 0, 2 * sizeof(unsigned)));
  // test hook (no GPU fault, no hang): the barrier expects one CTA more than is
  // launched, so every wait runs out after a short bounded spin
  const char* t = getenv("DG_TEST_BARRIER_TIMEOUT");
  if (t && atoi(t) > 0) {
    c->extra_arrivals = 1;
    c->spin_limit = 20000;
  }
  return DG_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int dg_num_planes(const dg_config* cfg) {
  if (validate(cfg)) return -1;
  return nplanes_of(cfg->eq, cfg->dim);
}

static dg_status init_common(const dg_config* cfgs, int nprob, void* stream, dg_ctx** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  if (!cfgs || nprob < 1) return fail(nullptr, DG_EINVAL, "need at least one configuration");
  for (int i = 0; i < nprob; ++i) {
    const char* m = validate(&cfgs[i]);
    if (m) return fail(nullptr, DG_EINVAL, "configuration %d: %s", i, m);
    const dg_config& a = cfgs[0];
    const dg_config& b = cfgs[i];
    if (b.eq != a.eq || b.dim != a.dim || b.precision != a.precision || b.gamma != a.gamma ||
        b.cfl != a.cfl || b.limiter != a.limiter || b.riemann != a.riemann ||
        b.integrator != a.integrator || b.face_points != a.face_points)
      return fail(nullptr, DG_EINVAL,
                  "batched problems must share eq, dim, precision, gamma, cfl, limiter, riemann, "
                  "integrator, face_points");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, DG_ECUDA, "no CUDA device available");
  }
  dg_ctx* c = new dg_ctx();
  const dg_config& a = cfgs[0];
  c->eq = a.eq; c->dim = a.dim; c->fp32 = a.precision == DG_FP32; c->limiter = a.limiter;
  c->gamma = a.gamma; c->cfl = a.cfl; c->ckpt_every = a.ckpt_every;
  c->integrator = a.integrator;
  // MUSCL-Hancock: 0 or 1 = the face-centroid rule; SSP-RK2: always the Gauss rule
  c->face_points = a.integrator == DG_MUSCL_HANCOCK && a.face_points != 2 ? 1 : 2;
  c->nplanes = nplanes_of(a.eq, a.dim);
  build_plane_map(c);
  c->stream = (cudaStream_t)stream;
  c->launch_stream = c->stream;
  if (const char* cap = getenv("DG_TEST_MAX_CTAS")) c->max_ctas = std::max(0, atoi(cap));
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(nullptr, DG_ECUDA, "could not create the capture stream");
  }
  size_t plane_off = 0;
  for (int i = 0; i < nprob; ++i) {
    Prob p;
    p.cfg = cfgs[i];
    p.nx = cfgs[i].n[0];
    p.ny = cfgs[i].n[1];
    p.nz = cfgs[i].dim == 3 ? cfgs[i].n[2] : 1;
    p.ncell = (long)p.nx * p.ny * p.nz;
    p.dx = cfgs[i].box[0] / p.nx;
    p.dy = cfgs[i].box[1] / p.ny;
    p.dz = cfgs[i].dim == 3 ? cfgs[i].box[2] / p.nz : 1.0;
    p.plane_off = plane_off;
    plane_off += (size_t)c->nplanes * p.ncell;
    c->ncell_total += p.ncell;
    c->probs.push_back(p);
  }
  dg_status s = alloc_ctx(c);
  if (s == DG_OK && nprob > 1 && c->dim == 2 && c->integrator == DG_SSPRK2) s = build_batch(c);
  if (s != DG_OK) {
    g_err = c->err;
    dg_destroy(c);
    return s;
  }
  *out = c;
  return DG_OK;
}

dg_status dg_init(const dg_config* cfg, void* cuda_stream, dg_ctx** out) {
  return init_common(cfg, 1, cuda_stream, out);
}

dg_status dg_init_batch(const dg_config* cfgs, int nprob, void* cuda_stream, dg_ctx** out) {
  return init_common(cfgs, nprob, cuda_stream, out);
}

void dg_destroy(dg_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_graphs(c);
  for (auto& e : c->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  adjoint_free(c->adj);
  for (int b = 0; b < 3; ++b) {
    cudaFree(c->c0[b]);
    cudaFree(c->sl[b]);
  }
  cudaFree(c->scratch);
  cudaFree(c->ctl);
  cudaFree(c->totals_dev);
  for (int v = 0; v < 3; ++v) cudaFree(c->btab[v]);
  cudaFree(c->bar);
  cudaFree(c->phase_dev);
  if (c->ctl_host) cudaFreeHost(c->ctl_host);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

const char* dg_last_error(const dg_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

dg_status dg_set_state(dg_ctx* c, const double* coeffs, int on_device) {
  if (!c || !coeffs) return fail(c, DG_EINVAL, "null argument");
  c->err.clear();
  dg_status s = c->fp32 ? set_state_t<float>(c, coeffs, on_device)
                        : set_state_t<double>(c, coeffs, on_device);
  if (s != DG_OK) return s;
  s = reset_ctl_and_cfl(c);
  if (s != DG_OK) return s;
  adjoint_reset(c->adj);
  c->state_set = true;
  s = check_err(c);
  if (s != DG_OK) return s;
  return autotune(c);
}

dg_status dg_get_state(dg_ctx* c, double* coeffs, int on_device) {
  if (!c || !coeffs) return fail(c, DG_EINVAL, "null argument");
  if (!c->state_set) return fail(c, DG_ESTATE, "no state has been set");
  return c->fp32 ? get_state_t<float>(c, coeffs, on_device) : get_state_t<double>(c, coeffs, on_device);
}

dg_status dg_step(dg_ctx* c, int nsteps, double dt_override, double* t_out) {
  if (!c) return DG_EINVAL;
  if (!c->state_set) return fail(c, DG_ESTATE, "no state has been set");
  if (nsteps < 0) return fail(c, DG_EINVAL, "nsteps must be >= 0");
  double dtov = dt_override > 0.0 ? dt_override : 0.0;
  // steps outside dg_record end the recorded trajectory: a later dg_record starts
  // a new one from the state these steps reach, and dg_adjoint has nothing to run
  // back over until then
  if (nsteps > 0) adjoint_reset(c->adj);
  int done = 0;
  if (!c->prof && nsteps >= 2) {
    cudaGraphExec_t ex;
    dg_status s = ensure_graph(c, dtov, &ex);
    if (s != DG_OK) return s;
    for (; done + 2 <= nsteps; done += 2) CK(c, cudaGraphLaunch(ex, c->stream));
  }
  for (; done < nsteps; ++done) {
    if (c->prof) CK(c, launch_step_profiled(c, c->cur, c->nxt, dtov));
    else CK(c, launch_step(c, c->cur, c->nxt, dtov));
    std::swap(c->cur, c->nxt);
  }
  if (t_out) {
    dg_status s = check_err(c);
    *t_out = c->ctl_host[0].t;
    return s;
  }
  return DG_OK;
}

dg_status dg_sync(dg_ctx* c) {
  if (!c) return DG_EINVAL;
  return check_err(c);
}

dg_status dg_get_times(dg_ctx* c, double* t, double* dt_next) {
  if (!c) return DG_EINVAL;
  dg_status s = read_ctl(c);
  if (s != DG_OK) return s;
  for (size_t p = 0; p < c->probs.size(); ++p) {
    if (t) t[p] = c->ctl_host[p].t;
    if (dt_next) {
      double vm = c->ctl_host[p].vmax_cur;
      dt_next[p] = vm > 0.0 ? c->cfl / vm : 0.0;
    }
  }
  return DG_OK;
}

dg_status dg_totals(dg_ctx* c, double* out) {
  if (!c || !out) return fail(c, DG_EINVAL, "null argument");
  if (!c->state_set) return fail(c, DG_ESTATE, "no state has been set");
  for (size_t ip = 0; ip < c->probs.size(); ++ip) {
    const Prob& p = c->probs[ip];
    CK(c, launch_totals(c->c0[c->cur] + p.c0_off, c->nv, p.ncell, c->scratch, c->totals_dev,
                        c->stream));
    double h[16];
    CK(c, cudaMemcpyAsync(h, c->totals_dev, c->nv * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    double V = p.dx * p.dy * (c->dim == 3 ? p.dz : 1.0);
    for (int v = 0; v < c->nv; ++v) out[ip * c->nv + v] = h[v] * V;
  }
  return DG_OK;
}

dg_status dg_divb(dg_ctx* c, double* out, int on_device) {
  if (!c || !out) return fail(c, DG_EINVAL, "null argument");
  if (c->eq != DG_MHD) return fail(c, DG_EINVAL, "div B is defined for MHD only");
  if (c->dim != 2) return fail(c, DG_EINVAL, "the Stokes div B estimate is implemented in 2D");
  if (!c->state_set) return fail(c, DG_ESTATE, "no state has been set");
  const Prob& p = c->probs[0];
  double* dst = on_device ? out : c->scratch;
  if (c->fp32) CK(c, launch_divb<float>(sbuf<float>(c, c->cur, p), p.nx, p.ny, p.dx, p.dy, dst, c->stream));
  else CK(c, launch_divb<double>(sbuf<double>(c, c->cur, p), p.nx, p.ny, p.dx, p.dy, dst, c->stream));
  if (!on_device)
    CK(c, cudaMemcpyAsync(out, c->scratch, p.ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return DG_OK;
}

dg_status dg_profile(dg_ctx* c, int enable) {
  if (!c) return DG_EINVAL;
  if (enable) {
    CK(c, cudaStreamSynchronize(c->stream));
    for (auto& e : c->evs) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    c->evs.clear();
#ifdef DG_PHASE_PROFILE
    const size_t bytes = 2 * kPhaseSlots * sizeof(unsigned long long);
    if (!c->phase_dev) CK(c, cudaMalloc(&c->phase_dev, bytes));
    CK(c, cudaMemset(c->phase_dev, 0, bytes));
#endif
  }
  c->prof = enable != 0;
  return DG_OK;
}

dg_status dg_phase_cycles(dg_ctx* c, double* cycles, int n) {
  if (!c || !cycles) return fail(c, DG_EINVAL, "null argument");
  if (n < 2 * kPhaseSlots) return fail(c, DG_EINVAL, "need room for %d counters", 2 * kPhaseSlots);
#ifdef DG_PHASE_PROFILE
  if (!c->phase_dev) return fail(c, DG_ESTATE, "enable profiling (dg_profile) first");
  unsigned long long h[2 * kPhaseSlots];
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaMemcpy(h, c->phase_dev, sizeof(h), cudaMemcpyDeviceToHost));
  for (int k = 0; k < 2 * kPhaseSlots; ++k) cycles[k] = (double)h[k];
  return DG_OK;
#else
  return fail(c, DG_EINVAL, "this library was built without phase profiling (DG_PHASE_PROFILE)");
#endif
}

dg_status dg_profile_read(dg_ctx* c, double ms[2], long long launches[2]) {
  if (!c || !ms || !launches) return DG_EINVAL;
  CK(c, cudaStreamSynchronize(c->stream));
  ms[0] = ms[1] = 0.0;
  launches[0] = launches[1] = 0;
  for (auto& e : c->evs) {
    float t = 0.0f;
    CK(c, cudaEventElapsedTime(&t, e.a, e.b));
    ms[e.kind] += t;
    // a batched 2D step is one launch; otherwise every problem is launched
    launches[e.kind] += c->batch2d && c->integrator == DG_SSPRK2 ? 1 : (long long)c->probs.size();
  }
  return DG_OK;
}

const char* dg_kernel_name(const dg_ctx* cc) {
  if (!cc) return "";
  dg_ctx* c = const_cast<dg_ctx*>(cc);
  const int v = c->variant < 0 ? 0 : c->variant;
  const char* prec = c->fp32 ? "fp32" : "fp64";
  char b[96];
  if (c->integrator == DG_MUSCL_HANCOCK && c->dim == 2)
    snprintf(b, sizeof(b), "mh2d_kernel %s %s %dpt", mh2d_variant_name(c->eq, c->fp32, v), prec,
             c->face_points);
  else if (c->integrator == DG_MUSCL_HANCOCK && c->eq == DG_MHD)
    snprintf(b, sizeof(b), "mh3m_kernel %s %s %dpt", mh3m_variant_name(c->fp32, v), prec,
             c->face_points);
  else if (c->integrator == DG_MUSCL_HANCOCK)
    snprintf(b, sizeof(b), "mh3d_kernel %s %s %dpt", mh3d_variant_name(c->fp32, v), prec,
             c->face_points);
  else if (c->batch2d)
    snprintf(b, sizeof(b), "batch2d_kernel %dx%d %s", batch2d_tile_x(c->fp32, v),
             batch2d_tile_y(c->fp32, v), prec);
  else if (c->dim == 2)
    snprintf(b, sizeof(b), "%s %s %s", v >= 3 ? "stage2d_tma_kernel" : "stage2d_kernel",
             stage2d_variant_name(c->eq, c->fp32, v), prec);
  else if (c->eq == DG_MHD)
    snprintf(b, sizeof(b), "stage3m_kernel %s %s", stage3m_variant_name(c->fp32, v), prec);
  else
    snprintf(b, sizeof(b), "stage3d_kernel %s %s", stage3d_variant_name(c->fp32, v), prec);
  c->kname = b;
  return c->kname.c_str();
}

double dg_stage_bytes(const dg_ctx* c, int stage) {
  if (!c) return 0.0;
  double per = (double)c->nv * 8.0 + (double)c->ns * (c->fp32 ? 4.0 : 8.0);
  if (c->integrator == DG_MUSCL_HANCOCK)  // one launch per step, reported as stage 2
    return (stage == 1 ? 0.0 : 2.0) * per * (double)c->ncell_total;
  if (c->batch2d)  // one fused launch per step, reported as stage 2
    return (stage == 1 ? 0.0 : 5.0) * per * (double)c->ncell_total;
  return (stage == 1 ? 2.0 : 3.0) * per * (double)c->ncell_total;
}

// ---------------------------------------------------------------------------
// adjoint entry points (implemented in dg_adjoint.cu)
// ---------------------------------------------------------------------------
dg_status dg_adjoint_step(dg_ctx* c, const double* lam_next, double* lam_prev, const double* u_n,
                          double dt) {
  if (!c || !lam_next || !lam_prev || !u_n) return fail(c, DG_EINVAL, "null argument");
  if (c->integrator != DG_SSPRK2) return fail(c, DG_EINVAL, "the adjoint is that of the SSP-RK2 step");
  if (c->limiter == 2)
    return fail(c, DG_EINVAL, "the adjoint covers the min/max limiter (limiter 0 or 1)");
  if (c->dim != 2 || c->probs.size() != 1)
    return fail(c, DG_EINVAL, "the adjoint is implemented for one 2D problem");
  if (!(dt > 0.0)) return fail(c, DG_EINVAL, "dt must be > 0");
  AdjointCall call;
  call.nx = c->probs[0].nx; call.ny = c->probs[0].ny;
  call.dx = c->probs[0].dx; call.dy = c->probs[0].dy;
  call.gamma = c->gamma; call.limiter = c->limiter; call.fp32 = c->fp32;
  call.eq = c->eq;
  call.stream = c->stream;
  std::string msg;
  dg_status s = adjoint_step(c->adj, call, u_n, lam_next, lam_prev, dt, msg);
  if (s != DG_OK) return fail(c, s, "%s", msg.c_str());
  return DG_OK;
}

dg_status dg_record(dg_ctx* c, int nsteps, double dt_override, double* t_out) {
  if (!c) return DG_EINVAL;
  if (!c->state_set) return fail(c, DG_ESTATE, "no state has been set");
  if (c->ckpt_every < 1) return fail(c, DG_EINVAL, "recording needs cfg.ckpt_every >= 1");
  if (c->integrator != DG_SSPRK2) return fail(c, DG_EINVAL, "the adjoint is that of the SSP-RK2 step");
  if (c->limiter == 2)
    return fail(c, DG_EINVAL, "the adjoint covers the min/max limiter (limiter 0 or 1)");
  if (c->dim != 2 || c->probs.size() != 1)
    return fail(c, DG_EINVAL, "the adjoint is implemented for one 2D problem");
  if (nsteps < 0) return fail(c, DG_EINVAL, "nsteps must be >= 0");
  const Prob& p = c->probs[0];
  std::string msg;
  // grow the store: checkpoints of the interchange state + time-step history
  dg_status s = adjoint_reserve(c->adj, c->nplanes, p.ncell, c->ckpt_every,
                                c->adj.nrec + nsteps, msg);
  if (s != DG_OK) return fail(c, s, "%s", msg.c_str());
  // point the control block at the history
  Ctl h;
  CK(c, cudaMemcpyAsync(&h, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  h.dt_hist = c->adj.dt_hist;
  h.hist_cap = c->adj.cap_steps;
  h.step = c->adj.nrec;
  CK(c, cudaMemcpyAsync(c->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
  const double dtov = dt_override > 0.0 ? dt_override : 0.0;
  for (int n = 0; n < nsteps;) {
    long long k = c->adj.nrec;
    if (k % c->ckpt_every == 0) {
      double* ck = c->adj.ckpt + (size_t)(k / c->ckpt_every) * c->nplanes * p.ncell;
      dg_status g = c->fp32 ? get_state_t<float>(c, ck, 1) : get_state_t<double>(c, ck, 1);
      if (g != DG_OK) return g;
    }
    // the steps up to the next checkpoint: pairs as the two-step graph, which
    // writes the same time-step history as single launches (the history index
    // lives in the control block on the device)
    const int run = (int)std::min<long long>(nsteps - n, c->ckpt_every - k % c->ckpt_every);
    int done = 0;
    if (!c->prof && run >= 2) {
      cudaGraphExec_t ex;
      dg_status g = ensure_graph(c, dtov, &ex);
      if (g != DG_OK) return g;
      for (; done + 2 <= run; done += 2) CK(c, cudaGraphLaunch(ex, c->stream));
    }
    for (; done < run; ++done) {
      CK(c, launch_step(c, c->cur, c->nxt, dtov));
      std::swap(c->cur, c->nxt);
    }
    c->adj.nrec += run;
    n += run;
  }
  if (nsteps > 0) c->adj.generation++;
  CK(c, cudaMemcpyAsync(&h, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  h.dt_hist = nullptr;
  h.hist_cap = 0;
  CK(c, cudaMemcpyAsync(c->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
  dg_status e = check_err(c);
  if (t_out) *t_out = c->ctl_host[0].t;
  return e;
}

long long dg_record_generation(const dg_ctx* c) { return c ? c->adj.generation : -1; }

dg_status dg_adjoint(dg_ctx* c, const double* lam_N, double* lam_0) {
  if (!c || !lam_N || !lam_0) return fail(c, DG_EINVAL, "null argument");
  if (c->adj.nrec == 0) return fail(c, DG_ESTATE, "no recorded steps (call dg_record first)");
  const Prob& p = c->probs[0];
  AdjointCall call;
  call.nx = p.nx; call.ny = p.ny; call.dx = p.dx; call.dy = p.dy;
  call.gamma = c->gamma; call.limiter = c->limiter; call.fp32 = c->fp32;
  call.eq = c->eq;
  call.stream = c->stream;
  std::string msg;
  dg_status s = adjoint_run(c->adj, call, c->nplanes, c->ckpt_every, lam_N, lam_0, msg);
  if (s != DG_OK) return fail(c, s, "%s", msg.c_str());
  return DG_OK;
}

}  // extern "C"
