// Boundary conditions of the jet (paper Sec. "Large Eddy Simulation
// Formulation": entrance, far field, exit, azimuthal periodicity, centerline),
// applied after every Runge-Kutta stage (Algorithm 2: Update(B.C., Visc.)).
// Order: far field (j = nj-1), then entrance (i = 0) and exit (i = ni-1),
// then the axis average (j = 0).  The ghost points are filled afterwards by
// the caller.
#include "jz_internal.cuh"

namespace jz {
namespace {

constexpr int kTPB = 128;

__device__ __forceinline__ void store_cons(const State& q, long long p, double rho, double u, double v, double w,
                                           double pr, double gm1) {
  q.q[0][p] = rho;
  q.q[1][p] = rho * u;
  q.q[2][p] = rho * v;
  q.q[3][p] = rho * w;
  q.q[4][p] = pr / gm1 + 0.5 * rho * (u * u + v * v + w * w);
}

// Riemann-invariant far field on j = nj-1, 1 <= i <= ni-2.
__global__ void k_farfield(Dims d, Consts c, GridDev g, State q) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int ni2 = d.ni - 2;
  if (t >= (long long)ni2 * d.nk) return;
  const int i = 1 + (int)(t % ni2), k = (int)(t / ni2);
  const int jb = d.nj - 1;
  const long long pb = pidx(d, i, jb, k), pi = pidx(d, i, jb - 1, k);
  const long long nb = (long long)d.nk * d.ni, sb = (long long)k * d.ni + i;
  const double sx = g.Sb[sb], sy = g.Sb[nb + sb], sz = g.Sb[2 * nb + sb];
  const double nm = sqrt(sx * sx + sy * sy + sz * sz);
  const double n[3] = {sx / nm, sy / nm, sz / nm};
  const double rho_i = q.q[0][pi];
  const double ui[3] = {q.q[1][pi] / rho_i, q.q[2][pi] / rho_i, q.q[3][pi] / rho_i};
  const double p_i = c.gm1 * (q.q[4][pi] - 0.5 * (q.q[1][pi] * ui[0] + q.q[2][pi] * ui[1] + q.q[3][pi] * ui[2]));
  const double a_i = sqrt(c.gamma * p_i / rho_i);
  const double un_i = ui[0] * n[0] + ui[1] * n[1] + ui[2] * n[2];
  const double Rp = un_i + 2.0 * a_i / c.gm1;
  const double Rm = -2.0 / c.gm1;
  const double un = 0.5 * (Rp + Rm);
  const double ab = 0.25 * c.gm1 * (Rp - Rm);
  const bool out = un > 0.0;
  double ut[3];
  for (int a = 0; a < 3; ++a) ut[a] = out ? ui[a] - un_i * n[a] : 0.0;
  const double s = out ? p_i / pow(rho_i, c.gamma) : c.p_inf;
  const double rho = pow(ab * ab / (c.gamma * s), 1.0 / c.gm1);
  const double pr = rho * ab * ab / c.gamma;
  store_cons(q, pb, rho, ut[0] + un * n[0], ut[1] + un * n[1], ut[2] + un * n[2], pr, c.gm1);
}

// Entrance (i = 0) and exit (i = ni-1) for 1 <= j <= nj-1, every k.
__global__ void k_inout(Dims d, Consts c, Inflow in, State q, const Scalars* sc, double alpha) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nj1 = d.nj - 1;
  const long long nface = (long long)nj1 * d.nk;
  // the 32 temporal factors sin(omega_f t + psi_mf) at t_n + alpha dt are the same at every
  // entrance node: one evaluation each per block
  __shared__ double sn[kNF];
  if (threadIdx.x < kNF) sn[threadIdx.x] = sin(in.omega[threadIdx.x % JZ_N_FREQ] * (sc->t + alpha * sc->dt) +
                                               in.psi[threadIdx.x]);
  __syncthreads();
  if (t >= 2 * nface) return;
  const bool exit_plane = t >= nface;
  const long long tt = exit_plane ? t - nface : t;
  const int j = 1 + (int)(tt % nj1), k = (int)(tt / nj1);
  if (!exit_plane) {
    // target: tanh profile + forcing at t_n + alpha dt
    const long long tab = (long long)k * d.nj + j;
    const long long plane = (long long)d.nk * d.nj;
    double f = 0.0;
    for (int mf = 0; mf < kNF; ++mf) f = f + in.amp[mf] * in.Gf[mf * plane + tab] * sn[mf];
    const double ut = in.u0[tab] + c.jet_mach * f;
    const long long p1 = pidx(d, 1, j, k), pb = pidx(d, 0, j, k);
    const double rho1 = q.q[0][p1];
    const double u1[3] = {q.q[1][p1] / rho1, q.q[2][p1] / rho1, q.q[3][p1] / rho1};
    const double p1v = c.gm1 * (q.q[4][p1] - 0.5 * (q.q[1][p1] * u1[0] + q.q[2][p1] * u1[1] + q.q[3][p1] * u1[2]));
    const double a1 = sqrt(c.gamma * p1v / rho1);
    const double Rm = u1[0] - 2.0 * a1 / c.gm1;
    const double Rp = ut + 2.0 * 1.0 / c.gm1;
    const double ub = 0.5 * (Rp + Rm);
    const double ab = 0.25 * c.gm1 * (Rp - Rm);
    const double rho_sub = pow(ab * ab / (c.gamma * c.p_inf), 1.0 / c.gm1);
    const double p_sub = rho_sub * ab * ab / c.gamma;
    const bool sup = ut >= 1.0;
    store_cons(q, pb, sup ? 1.0 : rho_sub, sup ? ut : ub, 0.0, 0.0, sup ? c.p_inf : p_sub, c.gm1);
  } else {
    const long long pi = pidx(d, d.ni - 2, j, k), pb = pidx(d, d.ni - 1, j, k);
    const double rho_i = q.q[0][pi];
    const double ui[3] = {q.q[1][pi] / rho_i, q.q[2][pi] / rho_i, q.q[3][pi] / rho_i};
    const double p_i = c.gm1 * (q.q[4][pi] - 0.5 * (q.q[1][pi] * ui[0] + q.q[2][pi] * ui[1] + q.q[3][pi] * ui[2]));
    const double eint = p_i / (c.gm1 * rho_i);
    const double pr = c.p_inf;
    const double rho = pr / (c.gm1 * eint);
    store_cons(q, pb, rho, ui[0], ui[1], ui[2], pr, c.gm1);
  }
}

// Axis j = 0: the ring j = 1 averaged over the azimuth, one block per i.
__global__ void k_axis(Dims d, State q) {
  const int i = blockIdx.x;
  double s[5] = {0, 0, 0, 0, 0};
  for (int k = threadIdx.x; k < d.nk; k += blockDim.x) {
    const long long p = pidx(d, i, 1, k);
    for (int m = 0; m < 5; ++m) s[m] += q.q[m][p];
  }
  __shared__ double red[5][kTPB / 32];
  for (int m = 0; m < 5; ++m) {
    double x = s[m];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[m][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  double mean[5];
  for (int m = 0; m < 5; ++m) {
    double x = 0.0;
    for (int w = 0; w < kTPB / 32; ++w) x += red[m][w];
    mean[m] = x / d.nk;
  }
  for (int k = threadIdx.x; k < d.nk; k += blockDim.x) {
    const long long p = pidx(d, i, 0, k);
    for (int m = 0; m < 5; ++m) q.q[m][p] = mean[m];
  }
}

struct Phases {
  double phi[kNF];
};

// Entrance tables at i = 0: u0 = U_j/2 [1 + tanh((0.5 - r)/(2 theta))] and
// Gf[m][f] = g(r) cos(m theta + phi_mf), g(r) = exp(-((r - 0.5)/0.1)^2),
// with r and theta from the node coordinates.
__global__ void k_build_inflow(Dims d, Consts c, GridDev g, double* u0, double* Gf, Phases ph) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)d.nj * d.nk) return;
  const double y = g.Xin[t], z = g.Xin[(long long)d.nj * d.nk + t];   // t = k nj + j
  const double r = sqrt(y * y + z * z);
  const double th = atan2(z, y);
  u0[t] = 0.5 * c.jet_mach * (1.0 + tanh((0.5 - r) / (2.0 * c.theta_mom)));
  const double x = (r - 0.5) / 0.1;
  const double gr = exp(-(x * x));
  const long long plane = (long long)d.nk * d.nj;
  for (int m = 0; m < JZ_N_MODES; ++m)
    for (int f = 0; f < JZ_N_FREQ; ++f) {
      const int mf = m * JZ_N_FREQ + f;
      Gf[mf * plane + t] = gr * cos(m * th + ph.phi[mf]);
    }
}

}  // namespace

cudaError_t bc_farfield(const Dims& d, const Consts& c, const GridDev& g, const State& q, cudaStream_t st) {
  const long long nf = (long long)(d.ni - 2) * d.nk;
  k_farfield<<<blocks_for(nf, kTPB), kTPB, 0, st>>>(d, c, g, q);
  return cudaGetLastError();
}

cudaError_t bc_inout(const Dims& d, const Consts& c, const Inflow& in, const State& q, const Scalars* sc,
                     double alpha, cudaStream_t st) {
  const long long nio = 2LL * (d.nj - 1) * d.nk;
  k_inout<<<blocks_for(nio, kTPB), kTPB, 0, st>>>(d, c, in, q, sc, alpha);
  return cudaGetLastError();
}

cudaError_t bc_axis(const Dims& d, const State& q, cudaStream_t st) {
  k_axis<<<d.ni, kTPB, 0, st>>>(d, q);
  return cudaGetLastError();
}

cudaError_t build_inflow(const Dims& d, const Consts& c, const GridDev& g, const jz_params& p, Inflow& in,
                         cudaStream_t st) {
  Phases ph;
  for (int mf = 0; mf < kNF; ++mf) {
    ph.phi[mf] = p.forcing_phi[mf];
    in.amp[mf] = p.forcing_amp[mf];
    in.psi[mf] = p.forcing_psi[mf];
  }
  for (int f = 0; f < JZ_N_FREQ; ++f) in.omega[f] = 2.0 * 3.141592653589793 * p.strouhal[f] * p.jet_mach;
  const long long n = (long long)d.nj * d.nk;
  k_build_inflow<<<blocks_for(n, kTPB), kTPB, 0, st>>>(d, c, g, in.u0, in.Gf, ph);
  return cudaGetLastError();
}

}  // namespace jz
