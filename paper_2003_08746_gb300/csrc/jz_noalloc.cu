// Allocation-free residual: jz_residual_noalloc.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: code whose
// device memory is owned by another allocator under a fixed budget (a
// framework's memory pool, an embedded or shared-GPU deployment), and
// latency-critical loops that cannot afford the implicit device-wide
// synchronisation of cudaFree or the first-touch cost of a fresh
// allocation.  For them this file provides one entry point that evaluates
// the FP64 residual (the four FP64 stage passes of jz_stage64.cu) with its
// scratch in a fixed device array that exists for the life of the library.
//
// The scratch is the file-scope array below.  In host code its name is only
// a host-side stand-in: the device address is looked up with
// cudaGetSymbolAddress, once per device, by the first call made on that
// device (with that device current); the first call should therefore come
// before any stream capture.  Every call on a device shares the array, so
// calls whose kernels overlap on the GPU (other streams, other host
// threads) race with each other; order them on one stream.  The array is
// charged on every device where this file's module is loaded: with CUDA's
// lazy module loading (the default since CUDA 12.2) when the first call
// looks up its address on that device, with eager loading when the
// library's context is created there.
#include <mutex>

#include "jz_internal.cuh"

namespace jz {
namespace {

constexpr size_t kScratchBytes = JZ_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr size_t kHeader = 256;          // Scalars block, 256-byte aligned

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Device of a device (or managed) pointer; -1 for host memory or an unknown pointer.  The
// caller has checked that no earlier error is pending, so an error raised by the probe itself
// is the only one cleared here.
int device_of(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

}  // namespace
}  // namespace jz

extern "C" int jz_residual_noalloc(const jz_grid* g, const jz_params* p, const double* q, double* rhs,
                                   void* stream) {
  using namespace jz;
  if (!g || !p || !q || !rhs) return set_error(JZ_ERR_ARG, "jz_residual_noalloc: NULL argument");
  Dims d;
  GridDev gd;
  if (!grid_view(g, &d, &gd)) return set_error(JZ_ERR_STATE, "jz_residual_noalloc: metrics not computed");
  if (gd.compact) return set_error(JZ_ERR_STATE, "jz_residual_noalloc: the grid is compact (FP32 metrics only)");
  if (p->precision != JZ_PREC_FP64)
    return set_error(JZ_ERR_ARG, "jz_residual_noalloc: only the FP64 form is available");
  if (!(p->gamma > 1.0) || !(p->Re > 0.0) || !(p->Pr > 0.0) || !(p->Pr_sgs > 0.0) || !(p->T_ref_K > 0.0) ||
      !(p->sigma > 0.0 && p->sigma < 1.0))
    return set_error(JZ_ERR_ARG, "jz_residual_noalloc: parameter out of range");
  // an error left by the caller's earlier work is reported, not cleared by the probes below
  cudaError_t pend = cudaPeekAtLastError();
  if (pend != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof msg, "jz_residual_noalloc: a CUDA error from earlier work is pending: %s",
             cudaGetErrorString(pend));
    return set_error(JZ_ERR_CUDA, msg);
  }
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return set_error(JZ_ERR_CUDA, cudaGetErrorString(e));
  const int dq = device_of(q), dr = device_of(rhs), dg = device_of(gd.V);
  if (dq < 0 || dr < 0) return set_error(JZ_ERR_ARG, "jz_residual_noalloc: q and rhs must be device pointers");
  if (dq != cur || dr != cur || dg != cur) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "jz_residual_noalloc: q (device %d), rhs (device %d) and the grid (device %d) must all be on the "
             "current device %d", dq, dr, dg, cur);
    return set_error(JZ_ERR_ARG, msg);
  }
  // scratch: Scalars block, padded state (5 fields), stage work arrays (42 fields)
  const size_t need = kHeader + (size_t)47 * (size_t)d.Np * sizeof(double);
  if (need > kScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "jz_residual_noalloc: grid needs %zu bytes of scratch, the fixed maximum is %zu bytes "
             "(about %zu padded nodes)", need, kScratchBytes, (kScratchBytes - kHeader) / (47 * sizeof(double)));
    return set_error(JZ_ERR_ARG, msg);
  }
  void* base = nullptr;
  e = scratch_address(&base);
  if (e != cudaSuccess) return set_error(JZ_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scalars* sc = static_cast<Scalars*>(base);
  double* f = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kHeader);
  auto next = [&]() { double* r = f; f += d.Np; return r; };
  State qp{};
  for (int m = 0; m < 5; ++m) qp.q[m] = next();
  Work64 w;
  w.u = next(); w.v = next(); w.w = next(); w.T = next(); w.p = next(); w.mu = next();
  for (int dir = 0; dir < 3; ++dir) {
    w.Lam[dir] = next();
    w.nu[dir] = next();
    for (int m = 0; m < 5; ++m) {
      w.H[dir][m] = next();
      w.G[dir][m] = next();
    }
  }
  const Consts c = make_consts(*p);
  // Every scratch element a kernel reads is written earlier in this call;
  // only the scalar block is cleared (the previous call's values stay in the rest).
  e = cudaMemsetAsync(sc, 0, sizeof(Scalars), st);
  if (e == cudaSuccess) e = pack_real(d, qp.q, q, 5, st);
  if (e == cudaSuccess) e = ghost_fill(d, qp.q, 5, st);
  if (e == cudaSuccess) e = nodal64(d, c, gd, w, qp, st);
  if (e == cudaSuccess) e = viscous64(d, c, gd, w, qp, st);
  if (e == cudaSuccess) e = faces64(d, c, w, qp, st);
  if (e == cudaSuccess) e = update64(d, gd, w, qp, qp, qp, sc, 0.0, 0, rhs, st);
  if (e != cudaSuccess) return set_error(JZ_ERR_CUDA, cudaGetErrorString(e));
  return JZ_OK;
}
