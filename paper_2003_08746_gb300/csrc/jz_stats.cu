// Running time statistics of the axial velocity u_x = (rho u_x) / rho, the
// quantities of the paper's validation (Sec. "Validation": time-averaged axial
// velocity on the centreline and in radial profiles at fixed x/D, axial
// velocity rms, potential-core length).
//
// Per real node the library keeps the running mean and the running sum of
// squared deviations (Welford's update: mean += (u - mean)/n,
// M2 += (u - mean_old)(u - mean_new)), which stays accurate when the
// fluctuations are many orders below the mean.  A sample reads rho and
// rho u_x and rewrites both accumulators: 48 bytes per node, coalesced along
// i, one sweep.  Its 8 FP64 instructions per node (reciprocal 3, product 1,
// Welford update 4) at 2 per SM per clock take longer than the 48 bytes at
// HBM speed, so the FP64 pipe bounds it.  The read-out averages mean and
// rms = sqrt(M2 / n) over the azimuth k for every (i, j).
#include "jz_internal.cuh"

namespace jz {
namespace {

constexpr int kTPB = 256;

__global__ void k_flow_sample(Dims d, const double* __restrict__ q0, const double* __restrict__ q1,
                              double* __restrict__ mean, double* __restrict__ m2, double inv_n) {
  const int i = blockIdx.x * kTPB + threadIdx.x;
  if (i >= d.ni) return;
  const int j = blockIdx.y, k = blockIdx.z;
  const long long p = pidx(d, i, j, k);
  const long long t = ((long long)k * d.nj + j) * d.ni + i;
  // one rounded product (never fused into the subtractions below, so that a single sample
  // leaves M2 exactly 0); the FP64 pipe, not HBM, bounds this kernel
  const double u = __dmul_rn(q1[p], rcp64(q0[p]));
  const double m = mean[t];
  const double dl = u - m;
  const double mn = m + dl * inv_n;
  mean[t] = mn;
  m2[t] += dl * (u - mn);
}

// One thread per (i, j); the loop over k reads consecutive i in consecutive threads.
__global__ void k_flow_final(Dims d, const double* __restrict__ mean, const double* __restrict__ m2, double inv_n,
                             double* __restrict__ out_mean, double* __restrict__ out_rms) {
  const long long plane = (long long)d.ni * d.nj;
  const long long t = blockIdx.x * (long long)kTPB + threadIdx.x;
  if (t >= plane) return;
  double sm = 0.0, sr = 0.0;
  for (int k = 0; k < d.nk; ++k) {
    const long long idx = k * plane + t;
    sm += mean[idx];
    sr += sqrt(m2[idx] * inv_n);
  }
  out_mean[t] = sm / d.nk;
  out_rms[t] = sr / d.nk;
}

}  // namespace

cudaError_t flow_sample(const Dims& d, const State& q, double* mean, double* m2, long long n, cudaStream_t st) {
  const dim3 grid((d.ni + kTPB - 1) / kTPB, d.nj, d.nk);
  k_flow_sample<<<grid, kTPB, 0, st>>>(d, q.q[0], q.q[1], mean, m2, 1.0 / (double)n);
  return cudaGetLastError();
}

cudaError_t flow_final(const Dims& d, const double* mean, const double* m2, long long n, double* out_mean,
                       double* out_rms, cudaStream_t st) {
  const long long plane = (long long)d.ni * d.nj;
  k_flow_final<<<(unsigned)((plane + kTPB - 1) / kTPB), kTPB, 0, st>>>(d, mean, m2, 1.0 / (double)n, out_mean,
                                                                         out_rms);
  return cudaGetLastError();
}

}  // namespace jz
