// Reductions: the CFL time step, the conservation totals and the state
// checks (minimum density and pressure, non-finite values).
#include "jz_internal.cuh"

namespace jz {
namespace {

constexpr int kTPB = 256;
constexpr int kStatBlocks = 1216;   // 8 x 152 SMs; fixed so the sums are reproducible

__device__ __forceinline__ double warp_max(double x) {
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// max over the advanced nodes of (lambda_xi + lambda_eta + lambda_zeta)/V.
__global__ void k_cfl_rate(Dims d, GridDev g, State q, Consts c, Scalars* sc) {
  Box b{0, 0, 0, d.ni, d.nj, d.nk};
  int i, j, k;
  double rate = 0.0;
  if (box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k) &&
      (d.topo != JZ_TOPO_JET || (i >= 1 && i <= d.ni - 2 && j >= 1 && j <= d.nj - 2))) {
    const long long p = pidx(d, i, j, k);
    rate = node_rate(g, c, p, q.q[0][p], q.q[1][p], q.q[2][p], q.q[3][p], q.q[4][p]);
  }
  __shared__ double red[kTPB / 32];
  rate = warp_max(rate);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rate;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < kTPB / 32 ? red[threadIdx.x] : 0.0;
    x = warp_max(x);
    // non-negative doubles order like their bit patterns
    if (threadIdx.x == 0 && x > 0.0)
      atomicMax(reinterpret_cast<unsigned long long*>(&sc->rate_max), (unsigned long long)__double_as_longlong(x));
  }
}

__global__ void k_set_dt(Consts c, Scalars* sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  sc->dt = c.dt_fixed > 0.0 ? c.dt_fixed : c.cfl / sc->rate_max;
  sc->rate_max = 0.0;
  sc->res_sum = 0.0;
}

__global__ void k_end_step(Scalars* sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  sc->t = sc->t + sc->dt;
}

// Totals sum Q_m V, min rho, min p, non-finite flag; grid-stride with a fixed
// grid, per-block partials reduced by one block in a fixed order.
__global__ void k_stats_partial(Dims d, GridDev g, State q, Consts c, double* part) {
  const long long n = (long long)d.ni * d.nj * d.nk;
  double tot[5] = {0, 0, 0, 0, 0};
  double mn_r = 1e300, mn_p = 1e300, bad = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % d.ni);
    const long long r = t / d.ni;
    const int j = (int)(r % d.nj), k = (int)(r / d.nj);
    const long long p = pidx(d, i, j, k);
    const double V = g.compact ? (double)g.Mf[p * kMF + MF_V] : g.V[p];
    double qq[5];
    for (int m = 0; m < 5; ++m) {
      qq[m] = q.q[m][p];
      tot[m] += qq[m] * V;
      if (!isfinite(qq[m])) bad = 1.0;
    }
    const double pr = c.gm1 * (qq[4] - 0.5 * (qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]) / qq[0]);
    mn_r = fmin(mn_r, qq[0]);
    mn_p = fmin(mn_p, pr);
    if (!(qq[0] > 0.0) || !(pr > 0.0)) bad = 1.0;
  }
  __shared__ double red[8][kTPB];
  red[0][threadIdx.x] = tot[0]; red[1][threadIdx.x] = tot[1]; red[2][threadIdx.x] = tot[2];
  red[3][threadIdx.x] = tot[3]; red[4][threadIdx.x] = tot[4];
  red[5][threadIdx.x] = mn_r; red[6][threadIdx.x] = mn_p; red[7][threadIdx.x] = bad;
  __syncthreads();
  for (int s = kTPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      for (int m = 0; m < 5; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + s];
      red[5][threadIdx.x] = fmin(red[5][threadIdx.x], red[5][threadIdx.x + s]);
      red[6][threadIdx.x] = fmin(red[6][threadIdx.x], red[6][threadIdx.x + s]);
      red[7][threadIdx.x] = fmax(red[7][threadIdx.x], red[7][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 8) part[blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_stats_final(const double* part, int nblk, Scalars* sc) {
  __shared__ double red[8][kTPB];
  double v[8] = {0, 0, 0, 0, 0, 1e300, 1e300, 0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    for (int m = 0; m < 5; ++m) v[m] += part[b * 8 + m];
    v[5] = fmin(v[5], part[b * 8 + 5]);
    v[6] = fmin(v[6], part[b * 8 + 6]);
    v[7] = fmax(v[7], part[b * 8 + 7]);
  }
  for (int m = 0; m < 8; ++m) red[m][threadIdx.x] = v[m];
  __syncthreads();
  for (int s = kTPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      for (int m = 0; m < 5; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + s];
      red[5][threadIdx.x] = fmin(red[5][threadIdx.x], red[5][threadIdx.x + s]);
      red[6][threadIdx.x] = fmin(red[6][threadIdx.x], red[6][threadIdx.x + s]);
      red[7][threadIdx.x] = fmax(red[7][threadIdx.x], red[7][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int m = 0; m < 5; ++m) sc->tot[m] = red[m][0];
    sc->min_rho = red[5][0];
    sc->min_p = red[6][0];
    sc->nonfinite = red[7][0] > 0.0 ? 1 : 0;
  }
}

}  // namespace

int stat_partial_count() { return kStatBlocks; }

cudaError_t cfl_rate(const Dims& d, const Consts& c, const GridDev& g, const State& q, Scalars* sc,
                     cudaStream_t st) {
  const long long nr = (long long)d.ni * d.nj * d.nk;
  k_cfl_rate<<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, g, q, c, sc);
  return cudaGetLastError();
}

cudaError_t set_dt(const Consts& c, Scalars* sc, int advance_time, cudaStream_t st) {
  if (advance_time)
    k_end_step<<<1, 32, 0, st>>>(sc);
  else
    k_set_dt<<<1, 32, 0, st>>>(c, sc);
  return cudaGetLastError();
}

cudaError_t stats_with(const Dims& d, const Consts& c, const GridDev& g, const State& q, Scalars* sc,
                       double* part, cudaStream_t st) {
  k_stats_partial<<<kStatBlocks, kTPB, 0, st>>>(d, g, q, c, part);
  k_stats_final<<<1, kTPB, 0, st>>>(part, kStatBlocks, sc);
  return cudaGetLastError();
}

}  // namespace jz
