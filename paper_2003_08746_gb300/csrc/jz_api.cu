// C ABI entry points (include/jz.h): handles, device memory, and the order of
// the kernels in a time step (Algorithm 2 main loop).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "jz_internal.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define JZ_CK(call)                                                                              \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(JZ_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                      \
  } while (0)

const double kAlpha[5] = {0.25, 1.0 / 6.0, 0.375, 0.5, 1.0};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Status for a failed device allocation: out of memory, or another CUDA error
// (no device, driver too old, a sticky error from an earlier fault).
int alloc_status(cudaError_t e) { return e == cudaErrorMemoryAllocation ? JZ_ERR_OOM : JZ_ERR_CUDA; }

// Device-side address of page-locked host memory (cudaHostAlloc / cudaHostRegister,
// mapped into the device's address space), or nullptr for other host memory.  Kernels
// read and write such buffers directly over the host link, with no staging copy.
void* pinned_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Owner of a list of device allocations.
struct DevMem {
  std::vector<void*> blocks;
  cudaStream_t user = nullptr;    // stream whose queued work may still use the blocks
  bool has_user = false;
  ~DevMem() { release(); }
  void used_by(cudaStream_t st) {
    user = st;
    has_user = true;
  }
  void release() {
    if (has_user && !blocks.empty()) cudaStreamSynchronize(user);
    for (void* b : blocks) cudaFree(b);
    blocks.clear();
  }
  // Zeroed on `st`, the stream that will use the buffer: a plain cudaMemset runs on
  // the legacy default stream, which a non-blocking stream does not wait for, so a
  // late memset could wipe data the owner's first kernels had already written.
  double* alloc(size_t n, cudaError_t& err, cudaStream_t st) {
    void* p = nullptr;
    err = cudaMalloc(&p, n * sizeof(double));
    if (err != cudaSuccess) return nullptr;
    blocks.push_back(p);
    err = cudaMemsetAsync(p, 0, n * sizeof(double), st);
    return static_cast<double*>(p);
  }
};

}  // namespace

struct jz_grid {
  jz::Dims d{};
  jz::GridDev g{};                // value-initialised: null pointers, compact = 0
  bool metrics = false;
  int nsolvers = 0;               // live solvers on this grid
  DevMem mem64;                   // FP64 coordinates and metrics (released by jz_grid_compact)
  DevMem mem;                     // surface copies; FP32 metrics of a compact grid
};

struct jz_solver {
  jz_grid* grid = nullptr;
  jz_params prm;
  jz::Consts c;
  cudaStream_t st = nullptr;
  jz::State qn{}, qa{}, qb{};
  jz::Work64 w{};
  bool fp32 = false;              // JZ_PREC_FP32FLUX form
  bool pair = false;              // JZ_PREC_FP64PAIR form (double-float stage passes)
  jz::DFMetrics mdf{};            // pair form: double-float copies of the metrics
  jz::QDF qdf{};                  // pair form: double-float copy of the stage input
  const float* Mf = nullptr;      // FP32 metric records (FP32-flux form; the grid's if compact)
  // FP32-flux form: TMA descriptors of the shadows of qn, qa, qb (the buffers swap roles, so a
  // descriptor is found by its shadow's address)
  struct TMap {
    alignas(64) unsigned char b[128];
  };
  TMap tmap[3];
  const float2* tkey[3] = {nullptr, nullptr, nullptr};
  const void* tmap_of(const jz::State& q) const {
    for (int i = 0; i < 3; ++i)
      if (tkey[i] == q.sh) return tmap[i].b;
    return nullptr;
  }
  int kchunk = 0;                 // k planes per CTA of the fused kernel
  bool rate_ready = false;        // a CFL rate of Q^n is in Scalars::rate_max
  jz::Scalars* sc = nullptr;
  jz::Inflow in{};
  double* part = nullptr;
  double* staging = nullptr;      // [5][N], allocated on first host transfer
  // flow statistics (jz_stats_*): per-node mean and M2, outputs [2][nj][ni]
  double* fs_mean = nullptr;
  double* fs_m2 = nullptr;
  double* fs_out = nullptr;
  long long fs_n = 0;
  int fs_every = 0;
  long long steps = 0;
  long long n_adv = 0;
  bool has_state = false;
  // per-kernel timing: an event after every kernel while profiling is on
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<cudaEvent_t> ev_marks;     // recorded, in stream order
  std::vector<int> ev_kind;              // kind of the kernel ending at each mark (-1: start)
  double prof_ms[JZ_NPROF] = {0};
  long long launches[JZ_NPROF] = {0};
  DevMem mem;
  void free_stats() {
    if (fs_mean || fs_m2 || fs_out) cudaStreamSynchronize(st);   // kernels may still use them
    if (fs_mean) cudaFree(fs_mean);
    if (fs_m2) cudaFree(fs_m2);
    if (fs_out) cudaFree(fs_out);
    fs_mean = fs_m2 = fs_out = nullptr;
    fs_n = 0;
    fs_every = 0;
  }
  // two-step CUDA graphs of jz_rk_step, keyed by the Q^n buffer they start from
  cudaStream_t cap_st = nullptr;           // private stream used only for capturing
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  const double* gkey[2] = {nullptr, nullptr};
  long long glaunch[2][JZ_NPROF] = {};     // kernel launches inside each graph, by kind
  bool graphs_off = false;
  ~jz_solver() {
    for (cudaGraphExec_t g : gexec)
      if (g) cudaGraphExecDestroy(g);
    if (cap_st) cudaStreamDestroy(cap_st);
    free_stats();
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ev_marks) cudaEventDestroy(e);
  }
};

namespace {

long long npts(const jz::Dims& d) { return (long long)d.ni * d.nj * d.nk; }

int ensure_staging(jz_solver* s) {
  if (s->staging) return JZ_OK;
  cudaError_t e;
  s->staging = s->mem.alloc(5 * (size_t)npts(s->grid->d), e, s->st);
  if (!s->staging) return fail(alloc_status(e), "staging buffer: %s", cudaGetErrorString(e));
  return JZ_OK;
}

// Copy a caller array [5][N] into the padded state q (ghosts filled).
int load_state(jz_solver* s, const double* src, jz::State& q) {
  const jz::Dims& d = s->grid->d;
  const double* dev = src;
  bool host = false;
  if (!is_device_ptr(src)) {
    host = true;
    dev = static_cast<const double*>(pinned_view(src));   // page-locked: the pack kernel reads it
    if (!dev) {                                           // pageable: staging copy
      int r = ensure_staging(s);
      if (r) return r;
      JZ_CK(cudaMemcpyAsync(s->staging, src, 5 * sizeof(double) * npts(d), cudaMemcpyHostToDevice, s->st));
      dev = s->staging;
    }
  }
  JZ_CK(jz::pack_real(d, q.q, dev, 5, s->st));
  JZ_CK(jz::ghost_fill(d, q.q, 5, s->st));
  if (s->fp32) JZ_CK(jz::shadow_refresh(d, s->c, q, 1, s->st));
  if (host) JZ_CK(cudaStreamSynchronize(s->st));           // the caller may reuse its host buffer
  return JZ_OK;
}

cudaEvent_t take_event(jz_solver* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Record a timing mark after a kernel of the given kind (kind -1: start mark).
int mark(jz_solver* s, int kind) {
  if (kind >= 0) s->launches[kind] += 1;
  if (!s->prof) return JZ_OK;
  cudaEvent_t e = take_event(s);
  if (!e) return fail(JZ_ERR_CUDA, "cudaEventCreate failed");
  JZ_CK(cudaEventRecord(e, s->st));
  s->ev_marks.push_back(e);
  s->ev_kind.push_back(kind);
  return JZ_OK;
}

#define JZ_RUN(kind, call)          \
  do {                              \
    JZ_CK(call);                    \
    int r_ = mark(s, (kind));       \
    if (r_) return r_;              \
  } while (0)

// cfl_first: stage 1 of a CFL step; the nodal pass reduces the rate of Q^n (Scalars::rate_max
// is 0 between FP64 steps) and the time step is set from it before the update.
int run_stage64(jz_solver* s, const jz::State& in, const jz::State& out, double alpha, int want_res,
                double* rhs_flat, bool cfl_first = false) {
  const jz::Dims& d = s->grid->d;
  const jz::GridDev& g = s->grid->g;
  if (s->pair) {
    JZ_RUN(JZ_PROF_NODAL, jz::nodal_df(d, s->c, s->mdf, s->w, s->qdf, in, s->st,
                                       cfl_first ? &s->sc->rate_max : nullptr));
    if (cfl_first) JZ_RUN(JZ_PROF_REDUCE, jz::set_dt(s->c, s->sc, 0, s->st));
    JZ_RUN(JZ_PROF_VISCOUS, jz::viscous_df(d, s->c, s->mdf, s->w, s->qdf, s->st));
    JZ_RUN(JZ_PROF_FACES, jz::faces_update_df(d, s->c, g, s->w, s->qdf, in, s->qn, out, s->sc, alpha, want_res,
                                              rhs_flat, s->st));
    return JZ_OK;
  }
  JZ_RUN(JZ_PROF_NODAL, jz::nodal64(d, s->c, g, s->w, in, s->st, cfl_first ? &s->sc->rate_max : nullptr));
  if (cfl_first) JZ_RUN(JZ_PROF_REDUCE, jz::set_dt(s->c, s->sc, 0, s->st));
  JZ_RUN(JZ_PROF_VISCOUS, jz::viscous64(d, s->c, g, s->w, in, s->st));
  JZ_RUN(JZ_PROF_FACES, jz::faces64(d, s->c, s->w, in, s->st));
  JZ_RUN(JZ_PROF_UPDATE, jz::update64(d, g, s->w, in, s->qn, out, s->sc, alpha, want_res, rhs_flat, s->st));
  return JZ_OK;
}

int run_step(jz_solver* s) {
  const jz::Dims& d = s->grid->d;
  const jz::GridDev& g = s->grid->g;
  const bool cfl = s->c.dt_fixed <= 0.0;
  // CFL rate of Q^n: the FP64 form reduces it in its stage-1 nodal pass, which forms the
  // spectral radii anyway; the FP32-flux form's stage 5 left it behind, and after
  // jz_set_state it is reduced here.
  if (s->fp32 || !cfl) {
    if (cfl && !s->rate_ready) JZ_RUN(JZ_PROF_REDUCE, jz::cfl_rate(d, s->c, g, s->qn, s->sc, s->st));
    JZ_RUN(JZ_PROF_REDUCE, jz::set_dt(s->c, s->sc, 0, s->st));
  }
  jz::State in = s->qn;
  for (int l = 0; l < 5; ++l) {
    jz::State out = (l % 2 == 0) ? s->qa : s->qb;
    int r = JZ_OK;
    if (s->fp32)
      JZ_RUN(JZ_PROF_FUSED32, jz::fused32(d, s->c, s->Mf, in, s->tmap_of(in), s->qn, out, s->sc, kAlpha[l], l == 0,
                                          l == 4 && cfl, nullptr, s->kchunk, s->st));
    else
      r = run_stage64(s, in, out, kAlpha[l], l == 0, nullptr, l == 0 && cfl);
    if (r) return r;
    if (d.topo == JZ_TOPO_JET) {
      JZ_RUN(JZ_PROF_BC, jz::bc_farfield(d, s->c, g, out, s->st));
      JZ_RUN(JZ_PROF_BC, jz::bc_inout(d, s->c, s->in, out, s->sc, kAlpha[l], s->st));
      JZ_RUN(JZ_PROF_BC, jz::bc_axis(d, out, s->st));
    }
    JZ_RUN(JZ_PROF_GHOST, jz::ghost_fill(d, out.q, 5, s->st));
    if (s->fp32) JZ_RUN(JZ_PROF_GHOST, jz::shadow_refresh(d, s->c, out, 0, s->st));
    in = out;
  }
  // Q^{n+1} is in qa (stage 5 wrote it); it becomes Q^n.
  jz::State t = s->qn;
  s->qn = s->qa;
  s->qa = t;
  JZ_RUN(JZ_PROF_REDUCE, jz::set_dt(s->c, s->sc, 1, s->st));
  s->steps += 1;
  s->rate_ready = s->fp32 && cfl;
  return JZ_OK;
}

// Two time steps replayed as one CUDA graph.  A step launches 27 (FP32-flux form) or 43
// (FP64 form) small kernels whose parameters never change between steps, except that the
// roles of the Q^n and stage buffers swap every step and come back after two; so two steps
// are captured once per starting buffer (on a private stream, nothing executes while
// capturing) and replayed with one launch.  Not used while profiling (events between
// kernels), while flow statistics are sampled, or before the first FP32-flux step has left a
// CFL rate.
// Any capture failure turns graphs off for the solver; the steps then run as plain launches.
int graph_two_steps(jz_solver* s, bool* done) {
  *done = false;
  if (s->graphs_off || s->prof || s->fs_every > 0) return JZ_OK;
  if (s->fp32 && s->c.dt_fixed <= 0.0 && !s->rate_ready) return JZ_OK;
  int slot = s->gkey[0] == s->qn.q[0] ? 0 : (s->gkey[1] == s->qn.q[0] ? 1 : -1);
  if (slot < 0) {
    slot = s->gexec[0] ? 1 : 0;
    if (s->gexec[slot]) {
      cudaGraphExecDestroy(s->gexec[slot]);
      s->gexec[slot] = nullptr;
      s->gkey[slot] = nullptr;
    }
    if (!s->cap_st && cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s->graphs_off = true;
      return JZ_OK;
    }
    // capture with the host bookkeeping saved, then restore it (nothing ran)
    const jz::State qn = s->qn, qa = s->qa, qb = s->qb;
    const long long steps = s->steps;
    const bool rate_ready = s->rate_ready;
    long long launches[JZ_NPROF];
    std::memcpy(launches, s->launches, sizeof launches);
    cudaStream_t user = s->st;
    s->st = s->cap_st;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->cap_st, cudaStreamCaptureModeThreadLocal);
    int r = JZ_OK;
    if (e == cudaSuccess) {
      r = run_step(s);
      if (r == JZ_OK) r = run_step(s);
      e = cudaStreamEndCapture(s->cap_st, &graph);
    }
    s->st = user;
    for (int k = 0; k < JZ_NPROF; ++k) s->glaunch[slot][k] = s->launches[k] - launches[k];
    std::memcpy(s->launches, launches, sizeof launches);
    s->qn = qn; s->qa = qa; s->qb = qb;
    s->steps = steps;
    s->rate_ready = rate_ready;
    if (e == cudaSuccess && r == JZ_OK && graph) e = cudaGraphInstantiate(&s->gexec[slot], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || r != JZ_OK || !s->gexec[slot]) {
      cudaGetLastError();
      s->gexec[slot] = nullptr;
      s->graphs_off = true;
      return JZ_OK;
    }
    s->gkey[slot] = s->qn.q[0];
  }
  JZ_CK(cudaGraphLaunch(s->gexec[slot], s->st));
  for (int k = 0; k < JZ_NPROF; ++k) s->launches[k] += s->glaunch[slot][k];
  s->steps += 2;
  s->rate_ready = s->fp32 && s->c.dt_fixed <= 0.0;
  *done = true;
  return JZ_OK;
}

int stats_sample(jz_solver* s) {
  s->fs_n += 1;
  JZ_RUN(JZ_PROF_STATS, jz::flow_sample(s->grid->d, s->qn, s->fs_mean, s->fs_m2, s->fs_n, s->st));
  return JZ_OK;
}

// ---- discrete adjoint: forward stages from an explicit Q^n --------------------------
// A pair-form solver advances the states in pair arithmetic (its reverse sweep also regenerates
// the intermediates the transposed kernels read with the pair nodal and viscous passes).
int fwd_stage(jz_solver* s, const jz::State& in, const jz::State& qn, const jz::State& out, int l) {
  const jz::Dims& d = s->grid->d;
  const jz::GridDev& g = s->grid->g;
  if (s->pair) {
    JZ_RUN(JZ_PROF_NODAL, jz::nodal_df(d, s->c, s->mdf, s->w, s->qdf, in, s->st));
    JZ_RUN(JZ_PROF_VISCOUS, jz::viscous_df(d, s->c, s->mdf, s->w, s->qdf, s->st));
    JZ_RUN(JZ_PROF_FACES, jz::faces_update_df(d, s->c, g, s->w, s->qdf, in, qn, out, s->sc, kAlpha[l], 0, nullptr,
                                              s->st));
  } else {
    JZ_RUN(JZ_PROF_NODAL, jz::nodal64(d, s->c, g, s->w, in, s->st));
    JZ_RUN(JZ_PROF_VISCOUS, jz::viscous64(d, s->c, g, s->w, in, s->st));
    JZ_RUN(JZ_PROF_FACES, jz::faces64(d, s->c, s->w, in, s->st));
    JZ_RUN(JZ_PROF_UPDATE, jz::update64(d, g, s->w, in, qn, out, s->sc, kAlpha[l], 0, nullptr, s->st));
  }
  if (d.topo == JZ_TOPO_JET) {
    JZ_RUN(JZ_PROF_BC, jz::bc_farfield(d, s->c, g, out, s->st));
    JZ_RUN(JZ_PROF_BC, jz::bc_inout(d, s->c, s->in, out, s->sc, kAlpha[l], s->st));
    JZ_RUN(JZ_PROF_BC, jz::bc_axis(d, out, s->st));
  }
  JZ_RUN(JZ_PROF_GHOST, jz::ghost_fill(d, out.q, 5, s->st));
  return JZ_OK;
}

// One time step in -> out (in, out distinct from the solver's stage buffers).
int fwd_step(jz_solver* s, const jz::State& in, const jz::State& out, double t, double dt) {
  JZ_CK(jz::set_time(s->sc, t, dt, s->st));
  const jz::State* src = &in;
  for (int l = 0; l < 5; ++l) {
    const jz::State& dst = l == 4 ? out : ((l % 2 == 0) ? s->qa : s->qb);
    int r = fwd_stage(s, *src, in, dst, l);
    if (r) return r;
    src = &dst;
  }
  return JZ_OK;
}

// One time step in -> out that leaves the four intermediate stage states in keep[0..3].
int fwd_step_keep(jz_solver* s, const jz::State& in, const jz::State& out, double t, double dt,
                  const jz::State keep[4]) {
  JZ_CK(jz::set_time(s->sc, t, dt, s->st));
  const jz::State* src = &in;
  for (int l = 0; l < 5; ++l) {
    const jz::State& dst = l == 4 ? out : keep[l];
    int r = fwd_stage(s, *src, in, dst, l);
    if (r) return r;
    src = &dst;
  }
  return JZ_OK;
}

int copy_state(jz_solver* s, const jz::State& dst, const jz::State& src) {
  const size_t bytes = sizeof(double) * s->grid->d.Np;
  for (int m = 0; m < 5; ++m) JZ_CK(cudaMemcpyAsync(dst.q[m], src.q[m], bytes, cudaMemcpyDeviceToDevice, s->st));
  return JZ_OK;
}

}  // namespace

namespace jz {

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

bool grid_view(const jz_grid* g, Dims* d, GridDev* dev) {
  if (!g || !g->metrics) return false;
  *d = g->d;
  *dev = g->g;
  return true;
}

}  // namespace jz

extern "C" {

const char* jz_last_error(void) { return g_err.c_str(); }

int jz_version(void) { return 1; }

int jz_create_grid(int ni, int nj, int nk, const double* xyz, const double* period, int topology,
                   jz_grid** out) {
  if (!out) return fail(JZ_ERR_ARG, "jz_create_grid: out is NULL");
  *out = nullptr;
  if (!xyz) return fail(JZ_ERR_ARG, "jz_create_grid: xyz is NULL");
  if (topology == JZ_TOPO_PERIODIC) {
    if (ni < 1 || nj < 1 || nk < 1) return fail(JZ_ERR_ARG, "periodic grid needs ni, nj, nk >= 1");
    if (!period) return fail(JZ_ERR_ARG, "periodic grid needs the period vectors");
  } else if (topology == JZ_TOPO_JET) {
    if (ni < 4 || nj < 4 || nk < 4 || (nk % 2))
      return fail(JZ_ERR_ARG, "jet grid needs ni >= 4, nj >= 4 and an even nk >= 4 (got %d x %d x %d)", ni, nj, nk);
  } else {
    return fail(JZ_ERR_ARG, "unknown topology %d", topology);
  }
  const jz::Dims d = jz::make_dims(ni, nj, nk, topology);
  if (d.Np > (1LL << 40)) return fail(JZ_ERR_ARG, "grid too large");
  jz_grid* g = new (std::nothrow) jz_grid;
  if (!g) return fail(JZ_ERR_OOM, "host allocation failed");
  g->d = d;
  cudaError_t e = cudaSuccess;
  double** slots[] = {&g->g.xyz[0], &g->g.xyz[1], &g->g.xyz[2], &g->g.S[0], &g->g.S[1], &g->g.S[2],
                      &g->g.S[3], &g->g.S[4], &g->g.S[5], &g->g.S[6], &g->g.S[7], &g->g.S[8],
                      &g->g.V, &g->g.invV, &g->g.Smag[0], &g->g.Smag[1], &g->g.Smag[2], &g->g.Delta};
  for (double** sl : slots) {
    *sl = g->mem64.alloc(d.Np, e, nullptr);
    if (!*sl || e != cudaSuccess) {
      delete g;
      return fail(alloc_status(e), "grid arrays: %s", cudaGetErrorString(e));
    }
  }
  g->g.Sb = g->mem.alloc(3 * (size_t)d.nk * d.ni, e, nullptr);
  if (e == cudaSuccess) g->g.Xin = g->mem.alloc(2 * (size_t)d.nk * d.nj, e, nullptr);
  if (e != cudaSuccess) {
    delete g;
    return fail(alloc_status(e), "grid surface arrays: %s", cudaGetErrorString(e));
  }
  const long long N = npts(d);
  // coordinates already on the device are padded in place; host ones go through a staging copy
  const double* src = xyz;
  double* tmp = nullptr;
  if (!is_device_ptr(xyz)) {
    e = cudaMalloc(&tmp, 3 * sizeof(double) * N);
    if (e != cudaSuccess) {
      delete g;
      return fail(alloc_status(e), "coordinate staging: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(tmp, xyz, 3 * sizeof(double) * N, cudaMemcpyHostToDevice);
    src = tmp;
  }
  if (e == cudaSuccess) e = jz::pad_coordinates(d, src, period, g->g, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) {
    delete g;
    return fail(JZ_ERR_CUDA, "jz_create_grid: %s", cudaGetErrorString(e));
  }
  *out = g;
  return JZ_OK;
}

int jz_destroy_grid(jz_grid* g) {
  if (!g) return fail(JZ_ERR_ARG, "jz_destroy_grid: NULL");
  if (g->nsolvers > 0) return fail(JZ_ERR_STATE, "jz_destroy_grid: %d solver(s) still use the grid", g->nsolvers);
  delete g;
  return JZ_OK;
}

int jz_compute_metrics(jz_grid* g) {
  if (!g) return fail(JZ_ERR_ARG, "jz_compute_metrics: NULL grid");
  const jz::Dims& d = g->d;
  DevMem scratch;
  double* s9[9];
  cudaError_t e;
  for (int i = 0; i < 9; ++i) {
    s9[i] = scratch.alloc(d.Np, e, nullptr);
    if (!s9[i]) return fail(alloc_status(e), "metric scratch: %s", cudaGetErrorString(e));
  }
  int* bad = nullptr;
  JZ_CK(cudaMalloc(&bad, sizeof(int)));
  scratch.blocks.push_back(bad);
  JZ_CK(cudaMemset(bad, 0, sizeof(int)));
  JZ_CK(jz::compute_metrics(d, g->g, s9, nullptr));
  JZ_CK(jz::check_volume(d, g->g, bad, nullptr));
  int nbad = 0;
  JZ_CK(cudaMemcpy(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost));
  if (nbad) return fail(JZ_ERR_ARG, "grid has %d advanced nodes with V <= 0", nbad);
  JZ_CK(jz::boundary_copies(d, g->g, nullptr));
  JZ_CK(cudaDeviceSynchronize());
  g->metrics = true;
  return JZ_OK;
}

int jz_grid_compact(jz_grid* g) {
  if (!g) return fail(JZ_ERR_ARG, "jz_grid_compact: NULL grid");
  if (!g->metrics) return fail(JZ_ERR_STATE, "jz_grid_compact: call jz_compute_metrics first");
  if (g->g.compact) return JZ_OK;
  if (g->nsolvers > 0) return fail(JZ_ERR_STATE, "jz_grid_compact: %d solver(s) still use the grid", g->nsolvers);
  const jz::Dims& d = g->d;
  cudaError_t e = cudaSuccess;
  float* Mf = reinterpret_cast<float*>(g->mem.alloc((size_t)d.Np * jz::kMF / 2, e, nullptr));
  if (e != cudaSuccess) return fail(alloc_status(e), "jz_grid_compact: %s", cudaGetErrorString(e));
  JZ_CK(jz::metrics_to_f32(d, g->g, Mf, nullptr));
  JZ_CK(cudaDeviceSynchronize());
  g->mem64.release();
  for (int c = 0; c < 3; ++c) g->g.xyz[c] = g->g.Smag[c] = nullptr;
  for (int c = 0; c < 9; ++c) g->g.S[c] = nullptr;
  g->g.V = g->g.invV = g->g.Delta = nullptr;
  g->g.Mf = Mf;
  g->g.compact = 1;
  return JZ_OK;
}

int jz_get_metrics(const jz_grid* g, double* out) {
  if (!g || !out) return fail(JZ_ERR_ARG, "jz_get_metrics: NULL argument");
  if (!g->metrics) return fail(JZ_ERR_STATE, "jz_get_metrics: metrics not computed");
  if (g->g.compact) return fail(JZ_ERR_STATE, "jz_get_metrics: the grid is compact (FP32 metrics only)");
  const jz::Dims& d = g->d;
  double* M[10];
  for (int i = 0; i < 9; ++i) M[i] = g->g.S[i];
  M[9] = g->g.V;
  const long long N = npts(d);
  const bool dev = is_device_ptr(out);
  double* dst = out;
  double* tmp = nullptr;
  if (!dev) {
    JZ_CK(cudaMalloc(&tmp, 10 * sizeof(double) * N));
    dst = tmp;
  }
  cudaError_t e = jz::unpack_real(d, M, dst, 10, nullptr);
  if (e == cudaSuccess && !dev) e = cudaMemcpy(out, tmp, 10 * sizeof(double) * N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(JZ_ERR_CUDA, "jz_get_metrics: %s", cudaGetErrorString(e));
  return JZ_OK;
}

int jz_create(jz_grid* g, const jz_params* p, void* stream, jz_solver** out) {
  if (!out) return fail(JZ_ERR_ARG, "jz_create: out is NULL");
  *out = nullptr;
  if (!g || !p) return fail(JZ_ERR_ARG, "jz_create: NULL grid or params");
  if (!g->metrics) return fail(JZ_ERR_STATE, "jz_create: call jz_compute_metrics first");
  if (!(p->gamma > 1.0) || !(p->Re > 0.0) || !(p->Pr > 0.0) || !(p->Pr_sgs > 0.0) || !(p->T_ref_K > 0.0) ||
      !(p->S1_K >= 0.0) || !(p->C_s >= 0.0) || !(p->kappa2 >= 0.0) || !(p->kappa4 >= 0.0) ||
      !(p->sigma > 0.0 && p->sigma < 1.0) || !(p->cfl > 0.0) || !(p->dt_fixed >= 0.0))
    return fail(JZ_ERR_ARG, "jz_create: parameter out of range");
  if (p->precision != JZ_PREC_FP64 && p->precision != JZ_PREC_FP32FLUX && p->precision != JZ_PREC_FP64PAIR)
    return fail(JZ_ERR_ARG, "jz_create: unknown precision %d", p->precision);
  if (g->g.compact && p->precision != JZ_PREC_FP32FLUX)
    return fail(JZ_ERR_STATE, "jz_create: a compact grid (FP32 metrics only) takes the FP32-flux form only");
  jz_solver* s = new (std::nothrow) jz_solver;
  if (!s) return fail(JZ_ERR_OOM, "host allocation failed");
  s->grid = g;
  s->prm = *p;
  s->c = jz::make_consts(*p);
  s->st = static_cast<cudaStream_t>(stream);
  const jz::Dims& d = g->d;
  cudaError_t e = cudaSuccess;
  auto A = [&](double*& dst, size_t n) {
    if (e != cudaSuccess) return;
    dst = s->mem.alloc(n, e, s->st);
  };
  for (int m = 0; m < 5; ++m) {
    A(s->qn.q[m], d.Np);
    A(s->qa.q[m], d.Np);
    A(s->qb.q[m], d.Np);
  }
  s->fp32 = p->precision == JZ_PREC_FP32FLUX;
  float* own_mf = nullptr;
  if (s->fp32) {
    jz::State* qs[3] = {&s->qn, &s->qa, &s->qb};
    for (int i = 0; i < 3; ++i) {
      double* tmp = nullptr;
      A(tmp, 3 * (size_t)d.Np);           // three float2 (8-byte) arrays of Np
      qs[i]->sh = reinterpret_cast<float2*>(tmp);
      s->tkey[i] = qs[i]->sh;
    }
    if (g->g.compact) {
      s->Mf = g->g.Mf;                     // the grid's own records
    } else {
      double* tmp = nullptr;
      A(tmp, (size_t)d.Np * jz::kMF / 2);  // kMF floats per padded node
      own_mf = reinterpret_cast<float*>(tmp);
      s->Mf = own_mf;
    }
    // CTAs of 30 x 8 columns marching in k, the k range split into chunks.  Rule fitted to
    // chunk-count sweeps over eight workloads (box 32x24x16 to jet 1000x400x500): about 32
    // planes per CTA, but at least two waves of CTAs over the resident slots (small grids are
    // latency-bound: more, shorter CTAs win even with the 3 priming planes each) and at most
    // thirty (large grids: longer CTAs amortise the priming).
    const int tx = jz::fused32_tile_x(), ty = jz::fused32_tile_y();
    const long long tiles = (long long)((d.ni + tx - 1) / tx) * ((d.nj + ty - 1) / ty);
    int slots = 304;
    if (jz::fused32_slots(&slots) != cudaSuccess) {
      cudaGetLastError();
      slots = 304;
    }
    long long best = std::max(1, (d.nk + 16) / 32);
    if (tiles * best < 2LL * slots) best = std::min<long long>(d.nk, (2LL * slots + tiles - 1) / tiles);
    if (tiles * best > 30LL * slots) best = std::max<long long>(1, 30LL * slots / tiles);
    s->kchunk = (d.nk + best - 1) / best;
  } else {
    s->pair = p->precision == JZ_PREC_FP64PAIR;
    if (s->pair) {
      auto P = [&](float2*& dst) {
        double* tmp = nullptr;
        A(tmp, d.Np);                      // one float2 (8 bytes) per padded node
        dst = reinterpret_cast<float2*>(tmp);
      };
      for (int c9 = 0; c9 < 9; ++c9) P(s->mdf.S[c9]);
      for (int c3 = 0; c3 < 3; ++c3) P(s->mdf.Smag[c3]);
      P(s->mdf.invV);
      P(s->mdf.Delta);
      for (int m = 0; m < 5; ++m) A(s->qdf.q[m], d.Np);
    }
    A(s->w.u, d.Np); A(s->w.v, d.Np); A(s->w.w, d.Np); A(s->w.T, d.Np); A(s->w.p, d.Np); A(s->w.mu, d.Np);
    for (int dir = 0; dir < 3; ++dir) {
      A(s->w.Lam[dir], d.Np);
      A(s->w.nu[dir], d.Np);
      for (int m = 0; m < 5; ++m) {
        A(s->w.H[dir][m], d.Np);
        // the face fluxes G of the FP64 faces and update passes; the pair form forms them on
        // chip (and its adjoint regenerates only the nodal and viscous intermediates)
        if (!s->pair) A(s->w.G[dir][m], d.Np);
      }
    }
  }
  double* scal = nullptr;
  A(scal, (sizeof(jz::Scalars) + 7) / 8);
  s->sc = reinterpret_cast<jz::Scalars*>(scal);
  A(s->part, 8 * (size_t)jz::stat_partial_count());
  if (d.topo == JZ_TOPO_JET) {
    A(s->in.u0, (size_t)d.nj * d.nk);
    A(s->in.Gf, (size_t)jz::kNF * d.nj * d.nk);
  }
  if (e != cudaSuccess) {
    delete s;
    return fail(alloc_status(e), "jz_create: device allocation failed: %s", cudaGetErrorString(e));
  }
  if (s->fp32) {
    for (int i = 0; i < 3; ++i) {
      e = jz::make_shadow_map(d, const_cast<float2*>(s->tkey[i]), s->tmap[i].b);
      if (e != cudaSuccess) {
        delete s;
        return fail(JZ_ERR_CUDA, "jz_create: TMA descriptor of the state shadow: %s", cudaGetErrorString(e));
      }
    }
  }
  if (s->pair) {
    e = jz::metrics_to_df(d, g->g, s->mdf, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
      delete s;
      return fail(JZ_ERR_CUDA, "jz_create: double-float metrics: %s", cudaGetErrorString(e));
    }
  }
  if (own_mf) {
    e = jz::metrics_to_f32(d, g->g, own_mf, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
      delete s;
      return fail(JZ_ERR_CUDA, "jz_create: FP32 metrics: %s", cudaGetErrorString(e));
    }
  }
  if (d.topo == JZ_TOPO_JET) {
    e = jz::build_inflow(d, s->c, g->g, *p, s->in, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
      delete s;
      return fail(JZ_ERR_CUDA, "jz_create: inflow tables: %s", cudaGetErrorString(e));
    }
  }
  s->n_adv = d.topo == JZ_TOPO_JET ? (long long)(d.ni - 2) * (d.nj - 2) * d.nk : npts(d);
  g->nsolvers += 1;
  *out = s;
  return JZ_OK;
}

int jz_destroy(jz_solver* s) {
  if (!s) return fail(JZ_ERR_ARG, "jz_destroy: NULL");
  cudaStreamSynchronize(s->st);
  s->grid->nsolvers -= 1;
  delete s;
  return JZ_OK;
}

int jz_set_state(jz_solver* s, const double* q, double t) {
  if (!s || !q) return fail(JZ_ERR_ARG, "jz_set_state: NULL argument");
  int r = load_state(s, q, s->qn);
  if (r) return r;
  jz::Scalars h;
  std::memset(&h, 0, sizeof h);
  h.t = t;
  JZ_CK(cudaMemcpyAsync(s->sc, &h, sizeof h, cudaMemcpyHostToDevice, s->st));
  JZ_CK(cudaStreamSynchronize(s->st));
  s->steps = 0;
  s->rate_ready = false;
  s->has_state = true;
  return JZ_OK;
}

int jz_get_state(jz_solver* s, double* q) {
  if (!s || !q) return fail(JZ_ERR_ARG, "jz_get_state: NULL argument");
  if (!s->has_state) return fail(JZ_ERR_STATE, "jz_get_state: no state set");
  const jz::Dims& d = s->grid->d;
  if (is_device_ptr(q)) {
    JZ_CK(jz::unpack_real(d, s->qn.q, q, 5, s->st));
    return JZ_OK;
  }
  if (double* mapped = static_cast<double*>(pinned_view(q))) {   // page-locked: written directly
    JZ_CK(jz::unpack_real(d, s->qn.q, mapped, 5, s->st));
    JZ_CK(cudaStreamSynchronize(s->st));
    return JZ_OK;
  }
  int r = ensure_staging(s);
  if (r) return r;
  JZ_CK(jz::unpack_real(d, s->qn.q, s->staging, 5, s->st));
  JZ_CK(cudaMemcpyAsync(q, s->staging, 5 * sizeof(double) * npts(d), cudaMemcpyDeviceToHost, s->st));
  JZ_CK(cudaStreamSynchronize(s->st));
  return JZ_OK;
}

int jz_residual(jz_solver* s, const double* q, double* rhs) {
  if (!s || !q || !rhs) return fail(JZ_ERR_ARG, "jz_residual: NULL argument");
  const jz::Dims& d = s->grid->d;
  int r = load_state(s, q, s->qb);
  if (r) return r;
  const bool dev = is_device_ptr(rhs);
  double* dst = rhs;
  if (!dev) {
    r = ensure_staging(s);
    if (r) return r;
    dst = s->staging;
  }
  if (s->prof) {
    r = mark(s, -1);
    if (r) return r;
  }
  if (s->fp32) {
    JZ_RUN(JZ_PROF_FUSED32, jz::fused32(d, s->c, s->Mf, s->qb, s->tmap_of(s->qb), s->qb, s->qb, s->sc, 0.0, 0, 0,
                                        dst, s->kchunk, s->st));
  } else {
    r = run_stage64(s, s->qb, s->qb, 0.0, 0, dst);
    if (r) return r;
  }
  if (!dev) {
    JZ_CK(cudaMemcpyAsync(rhs, dst, 5 * sizeof(double) * npts(d), cudaMemcpyDeviceToHost, s->st));
    JZ_CK(cudaStreamSynchronize(s->st));
  }
  return JZ_OK;
}

int jz_rk_step(jz_solver* s, int nsteps, jz_step_stats* out) {
  if (!s) return fail(JZ_ERR_ARG, "jz_rk_step: NULL solver");
  if (nsteps < 0) return fail(JZ_ERR_ARG, "jz_rk_step: nsteps < 0");
  if (!s->has_state) return fail(JZ_ERR_STATE, "jz_rk_step: no state set");
  if (s->prof && nsteps > 0) {
    int r = mark(s, -1);
    if (r) return r;
  }
  for (int n = 0; n < nsteps;) {
    if (nsteps - n >= 2) {
      bool done = false;
      int r = graph_two_steps(s, &done);
      if (r) return r;
      if (done) {
        n += 2;
        continue;
      }
    }
    int r = run_step(s);
    if (r) return r;
    ++n;
    if (s->fs_every > 0 && s->steps % s->fs_every == 0) {
      r = stats_sample(s);
      if (r) return r;
    }
  }
  if (!out) return JZ_OK;
  const jz::Dims& d = s->grid->d;
  s->launches[JZ_PROF_REDUCE] += 2;
  JZ_CK(jz::stats_with(d, s->c, s->grid->g, s->qn, s->sc, s->part, s->st));
  jz::Scalars h;
  JZ_CK(cudaMemcpyAsync(&h, s->sc, sizeof h, cudaMemcpyDeviceToHost, s->st));
  JZ_CK(cudaStreamSynchronize(s->st));
  out->t = h.t;
  out->dt = h.dt;
  out->res_l2 = s->steps > 0 ? std::sqrt(h.res_sum / (double)s->n_adv) : 0.0;
  for (int m = 0; m < 5; ++m) out->totals[m] = h.tot[m];
  out->min_rho = h.min_rho;
  out->min_p = h.min_p;
  out->steps = s->steps;
  if (h.wait_timeout) return fail(JZ_ERR_CUDA, "a stage kernel's bounded wait for its TMA copy ran out");
  if (h.nonfinite) return fail(JZ_ERR_NONFINITE, "state holds NaN/Inf or non-positive density/pressure");
  return JZ_OK;
}

int jz_adjoint_step(jz_solver* s, const double* forcing_amps, int nsteps, int ckpt_every, double r_obs,
                    double* J_out, double* grad_out) {
  if (!s || !forcing_amps || !J_out || !grad_out) return fail(JZ_ERR_ARG, "jz_adjoint_step: NULL argument");
  if (nsteps < 1 || ckpt_every < 1) return fail(JZ_ERR_ARG, "jz_adjoint_step: nsteps and ckpt_every must be >= 1");
  if (s->fp32) return fail(JZ_ERR_ARG, "jz_adjoint_step: the adjoint is available for the FP64 form");
  s->rate_ready = false;     // the sweep below reduces its own (frozen) rate into the scalars
  const jz::Dims& d = s->grid->d;
  const jz::GridDev& g = s->grid->g;
  if (d.topo != JZ_TOPO_JET) return fail(JZ_ERR_ARG, "jz_adjoint_step: the observer functional needs a jet grid");
  if (!s->has_state) return fail(JZ_ERR_STATE, "jz_adjoint_step: no state set");
  if (!(r_obs > 0.0)) return fail(JZ_ERR_ARG, "jz_adjoint_step: r_obs must be > 0");
  // observer geometry from the node coordinates: r_j at (i = 0, k = 0), x_i at (j = 0, k = 0)
  std::vector<double> y(d.nj), z(d.nj), x(d.ni);
  const size_t pitch = sizeof(double) * d.Pi;
  JZ_CK(cudaMemcpy2D(y.data(), sizeof(double), g.xyz[1] + jz::pidx(d, 0, 0, 0), pitch, sizeof(double), d.nj,
                     cudaMemcpyDeviceToHost));
  JZ_CK(cudaMemcpy2D(z.data(), sizeof(double), g.xyz[2] + jz::pidx(d, 0, 0, 0), pitch, sizeof(double), d.nj,
                     cudaMemcpyDeviceToHost));
  JZ_CK(cudaMemcpy(x.data(), g.xyz[0] + jz::pidx(d, 0, 0, 0), sizeof(double) * d.ni, cudaMemcpyDeviceToHost));
  int j0 = -1;
  std::vector<double> rj(d.nj);
  for (int j = 0; j < d.nj; ++j) {
    rj[j] = std::sqrt(y[j] * y[j] + z[j] * z[j]);
    if (rj[j] <= r_obs) j0 = j;
  }
  if (j0 < 0 || j0 >= d.nj - 1) return fail(JZ_ERR_ARG, "jz_adjoint_step: r_obs = %g outside the grid", r_obs);
  const double beta = (r_obs - rj[j0]) / (rj[j0 + 1] - rj[j0]);
  std::vector<double> w(d.ni);
  const double wr = r_obs * (2.0 * 3.141592653589793 / d.nk);
  for (int i = 0; i < d.ni; ++i) {
    const double dx = i == 0 ? 0.5 * (x[1] - x[0])
                             : (i == d.ni - 1 ? 0.5 * (x[d.ni - 1] - x[d.ni - 2]) : 0.5 * (x[i + 1] - x[i - 1]));
    w[i] = wr * dx;
  }
  // device memory for this call (released after the stream's queued work, also on errors)
  DevMem mem;
  mem.used_by(s->st);
  cudaError_t e = cudaSuccess;
  auto A = [&](double*& dst, size_t n) {
    if (e != cudaSuccess) return;
    dst = mem.alloc(n, e, s->st);
  };
  auto AS = [&](jz::State& st) {
    for (int m = 0; m < 5; ++m) A(st.q[m], d.Np);
  };
  const int C = ckpt_every;
  const int nseg = (nsteps + C - 1) / C;
  double* wdev = nullptr;
  A(wdev, d.ni);
  jz::Adj64 a;
  for (int m = 0; m < 5; ++m) {
    A(a.lam[m], d.Np); A(a.qnbar[m], d.Np); A(a.acc[m], d.Np);
  }
  for (int dir = 0; dir < 3; ++dir) {
    A(a.ca2[dir], d.Np); A(a.ca4[dir], d.Np);
    A(a.lfh[dir], d.Np); A(a.nb0[dir], d.Np); A(a.nb1[dir], d.Np);
    A(a.cpm[dir], d.Np); A(a.c0[dir], d.Np); A(a.ubd[dir], d.Np);
    for (int n = 0; n < 4; ++n) A(a.G[n][dir], d.Np);
  }
  A(a.mub, d.Np); A(a.rhob, d.Np); A(a.abar, jz::kNF); A(a.J, 1);
  std::vector<jz::State> ck(nseg), seg(C + 1), stg(4);
  jz::State wa{}, wb{};
  for (auto& st : ck) AS(st);
  for (auto& st : seg) AS(st);
  for (auto& st : stg) AS(st);
  AS(wa); AS(wb);
  if (e != cudaSuccess) return fail(alloc_status(e), "jz_adjoint_step: device allocation failed: %s", cudaGetErrorString(e));
  // Where memory allows, the segment recompute keeps the four intermediate stage states of
  // every step, so that the reverse sweep does not recompute them step by step (one forward
  // step per step less).  Kept only if they take under half of the free device memory.
  std::vector<jz::State> kept;
  {
    size_t free_b = 0, total_b = 0;
    const size_t need = (size_t)C * 4 * 5 * sizeof(double) * (size_t)d.Np;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && need < free_b / 2) {
      kept.resize((size_t)C * 4);
      for (auto& st : kept) AS(st);
      if (e != cudaSuccess) {        // not enough after all: run without them
        cudaGetLastError();
        e = cudaSuccess;
        kept.clear();
      }
    } else {
      cudaGetLastError();
    }
  }
  JZ_CK(cudaMemcpyAsync(wdev, w.data(), sizeof(double) * d.ni, cudaMemcpyHostToDevice, s->st));
  // the solver's own time and last step are left as they were (the sweeps below set the
  // time of every step they recompute)
  jz::Scalars h0;
  JZ_CK(cudaMemcpyAsync(&h0, s->sc, sizeof h0, cudaMemcpyDeviceToHost, s->st));
  JZ_CK(cudaStreamSynchronize(s->st));
  struct RestoreTime {
    jz_solver* s;
    double t, dt;
    ~RestoreTime() { jz::set_time(s->sc, t, dt, s->st); }
  } restore_time{s, h0.t, h0.dt};
  // frozen time step and start time
  if (s->c.dt_fixed <= 0.0) JZ_RUN(JZ_PROF_REDUCE, jz::cfl_rate(d, s->c, g, s->qn, s->sc, s->st));
  JZ_RUN(JZ_PROF_REDUCE, jz::set_dt(s->c, s->sc, 0, s->st));
  jz::Scalars h;
  JZ_CK(cudaMemcpyAsync(&h, s->sc, sizeof h, cudaMemcpyDeviceToHost, s->st));
  JZ_CK(cudaStreamSynchronize(s->st));
  const double dt = h.dt, t0 = h.t;
  // forcing amplitudes of this evaluation (restored on return)
  double saved[jz::kNF];
  for (int f = 0; f < jz::kNF; ++f) {
    saved[f] = s->in.amp[f];
    s->in.amp[f] = forcing_amps[f];
  }
  struct Restore {
    jz_solver* s;
    double* v;
    ~Restore() {
      for (int f = 0; f < jz::kNF; ++f) s->in.amp[f] = v[f];
    }
  } restore{s, saved};
  // forward sweep with checkpoints; J accumulated on the device
  int r = copy_state(s, wa, s->qn);
  if (r) return r;
  for (int n = 0; n < nsteps; ++n) {
    if (n % C == 0) {
      r = copy_state(s, ck[n / C], wa);
      if (r) return r;
    }
    r = fwd_step(s, wa, wb, t0 + n * dt, dt);
    if (r) return r;
    JZ_RUN(JZ_PROF_ADJOINT, jz::observer(d, s->c, wb, wdev, j0, beta, dt, a, 0, s->st));
    std::swap(wa, wb);
  }
  // reverse sweep, one checkpoint segment at a time
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int n0 = sg * C, n1 = std::min(n0 + C, nsteps);
    r = copy_state(s, seg[0], ck[sg]);
    if (r) return r;
    for (int q = 0; q < n1 - n0; ++q) {
      r = kept.empty() ? fwd_step(s, seg[q], seg[q + 1], t0 + (n0 + q) * dt, dt)
                       : fwd_step_keep(s, seg[q], seg[q + 1], t0 + (n0 + q) * dt, dt, &kept[(size_t)q * 4]);
      if (r) return r;
    }
    for (int n = n1 - 1; n >= n0; --n) {
      const jz::State& Qn = seg[n - n0];
      const jz::State& Qn1 = seg[n - n0 + 1];
      const double tn = t0 + n * dt;
      JZ_RUN(JZ_PROF_ADJOINT, jz::observer(d, s->c, Qn1, wdev, j0, beta, dt, a, 1, s->st));
      // stage states of step n: kept by the segment recompute, or recomputed here
      const jz::State* sv = kept.empty() ? stg.data() : &kept[(size_t)(n - n0) * 4];
      const jz::State* st[6] = {&Qn, &sv[0], &sv[1], &sv[2], &sv[3], &Qn1};
      if (kept.empty()) {
        JZ_CK(jz::set_time(s->sc, tn, dt, s->st));
        for (int l = 0; l < 4; ++l) {
          r = fwd_stage(s, *st[l], Qn, *st[l + 1], l);
          if (r) return r;
        }
      }
      for (int l = 4; l >= 0; --l) {
        JZ_RUN(JZ_PROF_ADJOINT, jz::adj_bcs(d, s->c, g, s->in, *st[l + 1], a, tn + kAlpha[l] * dt, s->st));
        JZ_RUN(JZ_PROF_ADJOINT, s->pair ? jz::adj_update_df(d, g, a, kAlpha[l] * dt, s->st)
                                        : jz::adj_update(d, g, a, kAlpha[l] * dt, s->st));
        // the forward intermediates the transposed passes read, regenerated in the solver's form
        if (s->pair) {
          JZ_RUN(JZ_PROF_NODAL, jz::nodal_df(d, s->c, s->mdf, s->w, s->qdf, *st[l], s->st));
          JZ_RUN(JZ_PROF_VISCOUS, jz::viscous_df(d, s->c, s->mdf, s->w, s->qdf, s->st));
        } else {
          JZ_RUN(JZ_PROF_NODAL, jz::nodal64(d, s->c, g, s->w, *st[l], s->st));
          JZ_RUN(JZ_PROF_VISCOUS, jz::viscous64(d, s->c, g, s->w, *st[l], s->st));
        }
        JZ_RUN(JZ_PROF_ADJOINT, jz::adj_stage(d, s->c, g, s->w, *st[l], a, s->pair ? &s->mdf : nullptr,
                                              s->pair ? &s->qdf : nullptr, s->st));
      }
      JZ_RUN(JZ_PROF_ADJOINT, jz::adj_add_qn(d, a, s->st));
    }
  }
  double Jh = 0.0;
  JZ_CK(cudaMemcpyAsync(&Jh, a.J, sizeof(double), cudaMemcpyDeviceToHost, s->st));
  JZ_CK(cudaMemcpyAsync(grad_out, a.abar, sizeof(double) * jz::kNF, cudaMemcpyDeviceToHost, s->st));
  JZ_CK(cudaStreamSynchronize(s->st));
  *J_out = Jh;
  return JZ_OK;
}

int jz_profile(jz_solver* s, int enable) {
  if (!s) return fail(JZ_ERR_ARG, "jz_profile: NULL solver");
  s->prof = enable != 0;
  return JZ_OK;
}

int jz_profile_read(jz_solver* s, double* ms, long long* launches) {
  if (!s) return fail(JZ_ERR_ARG, "jz_profile_read: NULL solver");
  JZ_CK(cudaStreamSynchronize(s->st));
  for (size_t i = 1; i < s->ev_marks.size(); ++i) {
    const int kind = s->ev_kind[i];
    if (kind < 0) continue;
    float t = 0.f;
    JZ_CK(cudaEventElapsedTime(&t, s->ev_marks[i - 1], s->ev_marks[i]));
    s->prof_ms[kind] += t;
  }
  for (cudaEvent_t e : s->ev_marks) s->ev_pool.push_back(e);
  s->ev_marks.clear();
  s->ev_kind.clear();
  for (int k = 0; k < JZ_NPROF; ++k) {
    if (ms) ms[k] = s->prof_ms[k];
    if (launches) launches[k] = s->launches[k];
    s->prof_ms[k] = 0.0;
    s->launches[k] = 0;
  }
  return JZ_OK;
}

const char* jz_profile_name(int kind) {
  static const char* names[JZ_NPROF] = {"nodal", "viscous", "faces", "update", "bc", "ghost", "reduce",
                                        "fused32", "adjoint", "stats"};
  return (kind >= 0 && kind < JZ_NPROF) ? names[kind] : "";
}

}  // extern "C"

// ---- snapshots ---------------------------------------------------------------------
namespace {

constexpr char kSnapMagic[8] = {'J', 'Z', 'S', 'N', 'A', 'P', '0', '1'};
constexpr size_t kSnapChunk = 64u << 20;        // bytes per host transfer

struct SnapHeader {
  char magic[8];
  int32_t version, header_bytes;
  int32_t ni, nj, nk, topology, precision, flags;
  int64_t steps;
  double t, dt, rate, res_sum;
  uint64_t params_hash, data_hash;
  unsigned char pad[JZ_SNAPSHOT_HEADER_BYTES - 8 - 8 * 4 - 8 - 4 * 8 - 2 * 8];
};
static_assert(sizeof(SnapHeader) == JZ_SNAPSHOT_HEADER_BYTES, "snapshot header size");

constexpr uint64_t kFnvOffset = 1469598103934665603ull, kFnvPrime = 1099511628211ull;

// FNV-1a over 64-bit words (one step per word).
uint64_t fnv_words(uint64_t h, const void* p, size_t nwords) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < nwords; ++i) {
    uint64_t w;
    std::memcpy(&w, b + 8 * i, 8);
    h = (h ^ w) * kFnvPrime;
  }
  return h;
}

// The parameters that fix a step's result: every jz_params field except precision.
uint64_t params_hash(const jz_params& p) {
  return fnv_words(kFnvOffset, &p, offsetof(jz_params, precision) / sizeof(double));
}

struct FileCloser {
  FILE* f = nullptr;
  ~FileCloser() { if (f) std::fclose(f); }
};
struct PinnedHost {
  void* p = nullptr;
  ~PinnedHost() { if (p) cudaFreeHost(p); }
};

}  // namespace

int jz_save_snapshot(jz_solver* s, const char* path) {
  if (!s || !path) return fail(JZ_ERR_ARG, "jz_save_snapshot: NULL argument");
  if (!s->has_state) return fail(JZ_ERR_STATE, "jz_save_snapshot: no state set");
  const jz::Dims& d = s->grid->d;
  int r = ensure_staging(s);
  if (r) return r;
  JZ_CK(jz::unpack_real(d, s->qn.q, s->staging, 5, s->st));
  jz::Scalars h;
  JZ_CK(cudaMemcpyAsync(&h, s->sc, sizeof h, cudaMemcpyDeviceToHost, s->st));
  JZ_CK(cudaStreamSynchronize(s->st));
  SnapHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, kSnapMagic, 8);
  hd.version = 1;
  hd.header_bytes = JZ_SNAPSHOT_HEADER_BYTES;
  hd.ni = d.ni; hd.nj = d.nj; hd.nk = d.nk; hd.topology = d.topo;
  hd.precision = s->prm.precision;
  hd.flags = s->rate_ready ? 1 : 0;
  hd.steps = s->steps;
  hd.t = h.t; hd.dt = h.dt; hd.rate = h.rate_max; hd.res_sum = h.res_sum;
  hd.params_hash = params_hash(s->prm);
  FileCloser fc;
  fc.f = std::fopen(path, "wb");
  if (!fc.f) return fail(JZ_ERR_ARG, "jz_save_snapshot: cannot open '%s' for writing", path);
  // header first (data hash patched in at the end)
  if (std::fwrite(&hd, sizeof hd, 1, fc.f) != 1) return fail(JZ_ERR_ARG, "jz_save_snapshot: write failed");
  PinnedHost buf;
  JZ_CK(cudaMallocHost(&buf.p, 2 * kSnapChunk));
  const size_t total = 5 * sizeof(double) * (size_t)npts(d);
  const char* src = reinterpret_cast<const char*>(s->staging);
  uint64_t dh = kFnvOffset;
  for (size_t off = 0; off < total; off += kSnapChunk) {
    const size_t n = std::min(kSnapChunk, total - off);
    char* hb = static_cast<char*>(buf.p) + ((off / kSnapChunk) & 1) * kSnapChunk;
    JZ_CK(cudaMemcpyAsync(hb, src + off, n, cudaMemcpyDeviceToHost, s->st));
    JZ_CK(cudaStreamSynchronize(s->st));
    dh = fnv_words(dh, hb, n / 8);
    if (std::fwrite(hb, 1, n, fc.f) != n) return fail(JZ_ERR_ARG, "jz_save_snapshot: write failed");
  }
  hd.data_hash = dh;
  if (std::fseek(fc.f, 0, SEEK_SET) != 0 || std::fwrite(&hd, sizeof hd, 1, fc.f) != 1)
    return fail(JZ_ERR_ARG, "jz_save_snapshot: header rewrite failed");
  const int cerr = std::fclose(fc.f);
  fc.f = nullptr;
  if (cerr != 0) return fail(JZ_ERR_ARG, "jz_save_snapshot: close failed");
  return JZ_OK;
}

int jz_load_snapshot(jz_solver* s, const char* path) {
  if (!s || !path) return fail(JZ_ERR_ARG, "jz_load_snapshot: NULL argument");
  const jz::Dims& d = s->grid->d;
  FileCloser fc;
  fc.f = std::fopen(path, "rb");
  if (!fc.f) return fail(JZ_ERR_ARG, "jz_load_snapshot: cannot open '%s'", path);
  SnapHeader hd;
  if (std::fread(&hd, sizeof hd, 1, fc.f) != 1) return fail(JZ_ERR_ARG, "jz_load_snapshot: short header");
  if (std::memcmp(hd.magic, kSnapMagic, 8) != 0 || hd.version != 1 || hd.header_bytes != JZ_SNAPSHOT_HEADER_BYTES)
    return fail(JZ_ERR_ARG, "jz_load_snapshot: '%s' is not a version-1 snapshot", path);
  if (hd.ni != d.ni || hd.nj != d.nj || hd.nk != d.nk || hd.topology != d.topo)
    return fail(JZ_ERR_ARG, "jz_load_snapshot: snapshot grid %d x %d x %d (topology %d) does not match %d x %d x %d (%d)",
                hd.ni, hd.nj, hd.nk, hd.topology, d.ni, d.nj, d.nk, d.topo);
  if (hd.params_hash != params_hash(s->prm))
    return fail(JZ_ERR_ARG, "jz_load_snapshot: snapshot was written with different parameters");
  int r = ensure_staging(s);
  if (r) return r;
  PinnedHost buf;
  JZ_CK(cudaMallocHost(&buf.p, 2 * kSnapChunk));
  const size_t total = 5 * sizeof(double) * (size_t)npts(d);
  char* dst = reinterpret_cast<char*>(s->staging);
  uint64_t dh = kFnvOffset;
  for (size_t off = 0; off < total; off += kSnapChunk) {
    const size_t n = std::min(kSnapChunk, total - off);
    char* hb = static_cast<char*>(buf.p) + ((off / kSnapChunk) & 1) * kSnapChunk;
    // the copy queued from this half two chunks ago must be done before it is refilled
    JZ_CK(cudaStreamSynchronize(s->st));
    if (std::fread(hb, 1, n, fc.f) != n) return fail(JZ_ERR_ARG, "jz_load_snapshot: short file '%s'", path);
    dh = fnv_words(dh, hb, n / 8);
    JZ_CK(cudaMemcpyAsync(dst + off, hb, n, cudaMemcpyHostToDevice, s->st));
  }
  JZ_CK(cudaStreamSynchronize(s->st));
  if (dh != hd.data_hash) return fail(JZ_ERR_ARG, "jz_load_snapshot: data hash mismatch in '%s'", path);
  r = load_state(s, s->staging, s->qn);
  if (r) return r;
  jz::Scalars h;
  std::memset(&h, 0, sizeof h);
  h.t = hd.t;
  h.dt = hd.dt;
  h.res_sum = hd.res_sum;
  // a stored rate is the FP32-flux form's (the FP64 form reduces its own in stage 1 and keeps
  // Scalars::rate_max at 0 between steps)
  const bool rate_ok = (hd.flags & 1) && hd.precision == s->prm.precision && s->fp32;
  if (rate_ok) h.rate_max = hd.rate;
  JZ_CK(cudaMemcpyAsync(s->sc, &h, sizeof h, cudaMemcpyHostToDevice, s->st));
  JZ_CK(cudaStreamSynchronize(s->st));
  s->steps = hd.steps;
  s->rate_ready = rate_ok;
  s->has_state = true;
  return JZ_OK;
}

// ---- flow statistics -------------------------------------------------------------
extern "C" {

int jz_stats_begin(jz_solver* s, int every) {
  if (!s) return fail(JZ_ERR_ARG, "jz_stats_begin: NULL solver");
  if (every < 0) return fail(JZ_ERR_ARG, "jz_stats_begin: every < 0");
  const jz::Dims& d = s->grid->d;
  if (d.nj > 65535 || d.nk > 65535) return fail(JZ_ERR_ARG, "jz_stats_begin: nj and nk must be <= 65535");
  s->free_stats();
  const size_t N = (size_t)npts(d), P = (size_t)d.ni * d.nj;
  cudaError_t e = cudaMalloc(&s->fs_mean, N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->fs_m2, N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->fs_out, 2 * P * sizeof(double));
  if (e != cudaSuccess) {
    s->free_stats();
    return fail(alloc_status(e), "jz_stats_begin: %s", cudaGetErrorString(e));
  }
  JZ_CK(cudaMemsetAsync(s->fs_mean, 0, N * sizeof(double), s->st));
  JZ_CK(cudaMemsetAsync(s->fs_m2, 0, N * sizeof(double), s->st));
  s->fs_every = every;
  return JZ_OK;
}

int jz_stats_sample(jz_solver* s) {
  if (!s) return fail(JZ_ERR_ARG, "jz_stats_sample: NULL solver");
  if (!s->fs_mean) return fail(JZ_ERR_STATE, "jz_stats_sample: call jz_stats_begin first");
  if (!s->has_state) return fail(JZ_ERR_STATE, "jz_stats_sample: no state set");
  return stats_sample(s);
}

int jz_stats_read(jz_solver* s, double* mean, double* rms, long long* nsamples) {
  if (!s) return fail(JZ_ERR_ARG, "jz_stats_read: NULL solver");
  if (!s->fs_mean) return fail(JZ_ERR_STATE, "jz_stats_read: call jz_stats_begin first");
  if (nsamples) *nsamples = s->fs_n;
  if (!mean && !rms) return JZ_OK;
  if (s->fs_n == 0) return fail(JZ_ERR_STATE, "jz_stats_read: no sample taken");
  const jz::Dims& d = s->grid->d;
  const size_t P = (size_t)d.ni * d.nj;
  JZ_RUN(JZ_PROF_STATS, jz::flow_final(d, s->fs_mean, s->fs_m2, s->fs_n, s->fs_out, s->fs_out + P, s->st));
  double* outs[2] = {mean, rms};
  bool host = false;
  for (int a = 0; a < 2; ++a) {
    if (!outs[a]) continue;
    const bool dev = is_device_ptr(outs[a]);
    host = host || !dev;
    JZ_CK(cudaMemcpyAsync(outs[a], s->fs_out + a * P, P * sizeof(double),
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->st));
  }
  if (host) JZ_CK(cudaStreamSynchronize(s->st));
  return JZ_OK;
}

int jz_stats_end(jz_solver* s) {
  if (!s) return fail(JZ_ERR_ARG, "jz_stats_end: NULL solver");
  JZ_CK(cudaStreamSynchronize(s->st));
  s->free_stats();
  return JZ_OK;
}

int jz_check_math(double* rcp_max_rel, double* cbrt_max_rel, double* sqrt_max_rel) {
  if (!rcp_max_rel || !cbrt_max_rel || !sqrt_max_rel) return fail(JZ_ERR_ARG, "jz_check_math: NULL argument");
  double* dev = nullptr;
  JZ_CK(cudaMalloc(&dev, 3 * sizeof(double)));
  double h[3] = {0.0, 0.0, 0.0};
  cudaError_t e = jz::math_check(dev, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(h, dev, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(dev);
  if (e != cudaSuccess) return fail(JZ_ERR_CUDA, "jz_check_math: %s", cudaGetErrorString(e));
  *rcp_max_rel = h[0];
  *cbrt_max_rel = h[1];
  *sqrt_max_rel = h[2];
  return JZ_OK;
}

int jz_check_pair(double* max_rel9) {
  if (!max_rel9) return fail(JZ_ERR_ARG, "jz_check_pair: NULL argument");
  double* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 9 * sizeof(double));
  if (e != cudaSuccess) return fail(alloc_status(e), "jz_check_pair: %s", cudaGetErrorString(e));
  e = jz::df_check(d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(max_rel9, d, 9 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(JZ_ERR_CUDA, "jz_check_pair: %s", cudaGetErrorString(e));
  return JZ_OK;
}

int jz_check_wait(int* timed_out, double* milliseconds) {
  if (!timed_out || !milliseconds) return fail(JZ_ERR_ARG, "jz_check_wait: NULL argument");
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 16);
  if (e != cudaSuccess) return fail(alloc_status(e), "jz_check_wait: %s", cudaGetErrorString(e));
  int* dt = static_cast<int*>(buf);
  long long* dc = reinterpret_cast<long long*>(static_cast<char*>(buf) + 8);
  e = jz::wait_check(dt, dc, nullptr);
  int h_t = 0;
  long long h_c = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h_t, dt, sizeof h_t, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&h_c, dc, sizeof h_c, cudaMemcpyDeviceToHost);
  int clk_khz = 0, dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(JZ_ERR_CUDA, "jz_check_wait: %s", cudaGetErrorString(e));
  *timed_out = h_t;
  *milliseconds = clk_khz > 0 ? (double)h_c / (double)clk_khz : 0.0;
  return JZ_OK;
}

int jz_station_profile(const double* field, const double* x, int ni, int nj, double x0, double* out) {
  if (!field || !x || !out || ni < 2 || nj < 1) return fail(JZ_ERR_ARG, "jz_station_profile: bad argument");
  if (!(x0 >= x[0] && x0 <= x[ni - 1])) return fail(JZ_ERR_ARG, "jz_station_profile: x0 outside the axial range");
  int i1 = 0;
  while (x[i1] < x0) ++i1;
  if (i1 == 0) {
    for (int j = 0; j < nj; ++j) out[j] = field[(size_t)j * ni];
    return JZ_OK;
  }
  const int i0 = i1 - 1;
  const double w = (x0 - x[i0]) / (x[i1] - x[i0]);
  for (int j = 0; j < nj; ++j)
    out[j] = (1.0 - w) * field[(size_t)j * ni + i0] + w * field[(size_t)j * ni + i1];
  return JZ_OK;
}

int jz_potential_core(const double* axis, const double* x, int ni, double u_jet, double frac, double* x_core) {
  if (!axis || !x || !x_core || ni < 2) return fail(JZ_ERR_ARG, "jz_potential_core: bad argument");
  const double thr = frac * u_jet;
  for (int i = 0; i < ni; ++i) {
    if (axis[i] < thr) {
      if (i == 0) {
        *x_core = x[0];
      } else {
        const double w = (axis[i - 1] - thr) / (axis[i - 1] - axis[i]);
        *x_core = x[i - 1] + w * (x[i] - x[i - 1]);
      }
      return JZ_OK;
    }
  }
  *x_core = NAN;
  return JZ_OK;
}

}  // extern "C"
