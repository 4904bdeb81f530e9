// FP64 form of one Runge-Kutta stage (Algorithm 2: the steps from the inviscid
// flux to the update of the conserved variables with alpha_l), as four passes
// over the padded grid.
//
// The FP64 pipe of a GB300 runs at 1/64 of its FP32 rate (2 against 128 lanes
// per SM per clock), so this form is
// bound by FP64 arithmetic, not by HBM.  Each pass therefore computes every
// nodal or face quantity exactly once and hands it to the next pass through
// HBM (no halo recomputation); the extra traffic costs far less time than
// the FP64 operations it saves.
//
//  A  nodal     (all padded nodes): primitives u, v, w, p, T; Sutherland mu;
//               spectral radii and their anisotropic scaling Lambda_dir;
//               transformed inviscid fluxes E^dir = S^dir_j E_j.
//  B  viscous   (nodes within one layer of the real region): Cartesian
//               gradients by the chain rule, strain rate, Smagorinsky eddy
//               viscosity, stresses and heat flux; H^dir = E^dir - S^dir_j F_j
//               (in place over E^dir); pressure sensor nu_dir.
//  C  faces     Turkel-Vatsa dissipation flux d_{n+1/2} for each direction,
//               combined with the face average of H into the doubled total
//               face flux G_{n+1/2} = H_n + H_{n+1} - 2 d_{n+1/2}.
//  D  update    V RHS = sum_dir [delta_dir H^dir - (d_{n+1/2} - d_{n-1/2})]
//                     = (1/2) sum_dir (G_{n+1/2} - G_{n-1/2}),
//               Q^(l) = Q^n - alpha_l dt RHS on the advanced nodes.
#include "jz_internal.cuh"

namespace jz {
namespace {

constexpr int kTPB = 256;

__device__ __forceinline__ bool advanced(const Dims& d, int i, int j) {
  return d.topo != JZ_TOPO_JET || (i >= 1 && i <= d.ni - 2 && j >= 1 && j <= d.nj - 2);
}

// Anisotropic spectral radius lambda_d + lambda_d^(1-sigma) (lambda_e^sigma + lambda_f^sigma).
__device__ __forceinline__ void aniso(const Consts& c, const double lam[3], double Lam[3]) {
  double lo[3], hi[3];
  if (c.sigma_is_two_thirds) {
    for (int d = 0; d < 3; ++d) cbrt_pair64(lam[d], lo[d], hi[d]);
  } else {
    for (int d = 0; d < 3; ++d) {
      lo[d] = lam[d] > 0.0 ? pow(lam[d], 1.0 - c.sigma) : 0.0;
      hi[d] = lam[d] > 0.0 ? pow(lam[d], c.sigma) : 0.0;
    }
  }
  Lam[0] = lam[0] + lo[0] * (hi[1] + hi[2]);
  Lam[1] = lam[1] + lo[1] * (hi[0] + hi[2]);
  Lam[2] = lam[2] + lo[2] * (hi[0] + hi[1]);
}

// rate_max != nullptr (stage 1): also the CFL rate of the stage input Q^n over the advanced
// nodes, max of (lambda_xi + lambda_eta + lambda_zeta) / V, from the spectral radii this pass
// forms anyway (the same expressions as the stand-alone rate pass), reduced block-wise into
// *rate_max; the time step is set from it before the stage's update.
__global__ void __launch_bounds__(kTPB) k_nodal(Dims d, Consts c, GridDev g, Work64 w, State q, double* rate_max) {
  Box b{-kG, -kG, -kG, d.ni + 2 * kG, d.nj + 2 * kG, d.nk + 2 * kG};
  int i, j, k;
  double rate = 0.0;
  if (box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) {
    const long long p = pidx(d, i, j, k);
    const double rho = q.q[0][p], m1 = q.q[1][p], m2 = q.q[2][p], m3 = q.q[3][p], e = q.q[4][p];
    const double ir = rcp64(rho);                 // one reciprocal instead of four divisions
    const double u = m1 * ir, v = m2 * ir, ww = m3 * ir;
    const double pr = fma(-c.gm1_half, m1 * u + m2 * v + m3 * ww, c.gm1 * e);   // (gamma-1)(e - rho|u|^2/2)
    const double T = c.gamma * pr * ir;
    const double a = sqrt64(T);
    // Sutherland, eq. (sutherland), with T_inf = 1
    const double mu = c.mu_sut * (T * a) * rcp64(T + c.S_hat);
    w.u[p] = u; w.v[p] = v; w.w[p] = ww; w.T[p] = T; w.p[p] = pr; w.mu[p] = mu;
    double lam[3];
    for (int dir = 0; dir < 3; ++dir) {
      const double sx = g.S[3 * dir][p], sy = g.S[3 * dir + 1][p], sz = g.S[3 * dir + 2][p];
      const double U = sx * u + sy * v + sz * ww;
      lam[dir] = fabs(U) + a * g.Smag[dir][p];
      w.H[dir][0][p] = rho * U;
      w.H[dir][1][p] = m1 * U + pr * sx;
      w.H[dir][2][p] = m2 * U + pr * sy;
      w.H[dir][3][p] = m3 * U + pr * sz;
      w.H[dir][4][p] = (e + pr) * U;
    }
    if (rate_max && i >= 0 && i < d.ni && j >= 0 && j < d.nj && k >= 0 && k < d.nk && advanced(d, i, j))
      rate = ((lam[0] + lam[1]) + lam[2]) * g.invV[p];
    double Lam[3];
    aniso(c, lam, Lam);
    w.Lam[0][p] = Lam[0]; w.Lam[1][p] = Lam[1]; w.Lam[2][p] = Lam[2];
  }
  if (rate_max) {
    // block max -> one atomic per block (non-negative doubles order like their bits)
    __shared__ double redm[kTPB / 32];
    for (int o = 16; o > 0; o >>= 1) rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = rate;
    __syncthreads();
    if (threadIdx.x < 32) {
      double x = threadIdx.x < kTPB / 32 ? redm[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
      if (threadIdx.x == 0 && x > 0.0)
        atomicMax(reinterpret_cast<unsigned long long*>(rate_max), (unsigned long long)__double_as_longlong(x));
    }
  }
}

__global__ void __launch_bounds__(kTPB) k_viscous(Dims d, Consts c, GridDev g, Work64 w, State q) {
  Box b{-1, -1, -1, d.ni + 2, d.nj + 2, d.nk + 2};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const long long s[3] = {1, d.sj, d.sk};
  const double* f[4] = {w.u, w.v, w.w, w.T};
  double S[3][3];
  for (int dir = 0; dir < 3; ++dir)
    for (int cc = 0; cc < 3; ++cc) S[dir][cc] = g.S[3 * dir + cc][p];
  const double iV = g.invV[p];
  // G[n][j] = sum_dir S^dir_j (f_n[+dir] - f_n[-dir]); the gradient is h G with h = 1/(2V),
  // and h is applied to the few products below instead of to the nine metrics
  double G[4][3];
  for (int n = 0; n < 4; ++n) {
    double dd[3];
    for (int dir = 0; dir < 3; ++dir) dd[dir] = f[n][p + s[dir]] - f[n][p - s[dir]];
    for (int jj = 0; jj < 3; ++jj) G[n][jj] = S[0][jj] * dd[0] + S[1][jj] * dd[1] + S[2][jj] * dd[2];
  }
  const double h = 0.5 * iV;
  // strain rate s = h sym(G): s_ii = h G_ii, s_ij = (h/2) A_ij with A_ij = G_ij + G_ji, so
  //   |S| = sqrt(2 s:s) = h sqrt(2 sum G_ii^2 + sum_{i<j} A_ij^2)
  const double A12 = G[0][1] + G[1][0], A13 = G[0][2] + G[2][0], A23 = G[1][2] + G[2][1];
  const double Gd = G[0][0] + G[1][1] + G[2][2];
  const double DG = G[0][0] * G[0][0] + G[1][1] * G[1][1] + G[2][2] * G[2][2];
  const double AA = A12 * A12 + A13 * A13 + A23 * A23;
  const double mu = w.mu[p];
  const double csd = c.C_s * g.Delta[p];
  // Smagorinsky eddy viscosity rho (C_s Delta)^2 |S|
  const double mu_sgs = q.q[0][p] * (csd * csd) * h * sqrt64(fma(2.0, DG, AA));
  const double mt = mu + mu_sgs;
  // tau_ii = 2 mt (s_ii - div/3) = (mt/V) (G_ii - Gd/3);  tau_ij = 2 mt s_ij = (mt h) A_ij
  const double mV = mt * iV, mh = mt * h;
  const double kh = (mu * c.k_lam + mu_sgs * c.k_sgs) * h;   // k_eff h: heat flux k_eff h G_T
  const double d3 = Gd * (1.0 / 3.0);
  const double t11 = mV * (G[0][0] - d3), t22 = mV * (G[1][1] - d3), t33 = mV * (G[2][2] - d3);
  const double t12 = mh * A12, t13 = mh * A13, t23 = mh * A23;
  const double tau[3][3] = {{t11, t12, t13}, {t12, t22, t23}, {t13, t23, t33}};
  const double vel[3] = {w.u[p], w.v[p], w.w[p]};
  // Cartesian viscous flux in direction jj: [tau_1j, tau_2j, tau_3j, u_i tau_ij + k dT/dx_j]
  double F[3][4];
  for (int jj = 0; jj < 3; ++jj) {
    F[jj][0] = tau[0][jj];
    F[jj][1] = tau[1][jj];
    F[jj][2] = tau[2][jj];
    F[jj][3] = vel[0] * tau[0][jj] + vel[1] * tau[1][jj] + vel[2] * tau[2][jj] + kh * G[3][jj];
  }
  // H^dir -= S^dir_j F_j, as three fused multiply-adds onto the stored E^dir
  for (int dir = 0; dir < 3; ++dir)
    for (int m = 0; m < 4; ++m)
      w.H[dir][m + 1][p] = fma(-S[dir][2], F[2][m], fma(-S[dir][1], F[1][m], fma(-S[dir][0], F[0][m],
                                                                                 w.H[dir][m + 1][p])));
  // pressure sensor along each direction: |p+ - 2p + p-| / (p+ + 2p + p-)
  const double pc = w.p[p];
  for (int dir = 0; dir < 3; ++dir) {
    const double sum = w.p[p + s[dir]] + w.p[p - s[dir]];
    w.nu[dir][p] = fabs(fma(-2.0, pc, sum)) * rcp64(fma(2.0, pc, sum));
  }
}

__global__ void __launch_bounds__(kTPB) k_faces(Dims d, Consts c, Work64 w, State q) {
  Box b{-1, -1, -1, d.ni + 1, d.nj + 1, d.nk + 1};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const long long s[3] = {1, d.sj, d.sk};
  for (int dir = 0; dir < 3; ++dir) {
    const long long sd = s[dir];
    // the sensor maximum and the clamp at 0 compare bit patterns on the integer pipe (the
    // sensors are >= 0, and non-negative doubles order like their bits)
    const long long nu0 = __double_as_longlong(w.nu[dir][p]), nu1 = __double_as_longlong(w.nu[dir][p + sd]);
    const double eps2 = c.kappa2 * __longlong_as_double(nu0 >= nu1 ? nu0 : nu1);
    const double k4 = c.kappa4 - eps2;
    const double eps4 = __double_as_longlong(k4) > 0 ? k4 : 0.0;
    // d = L_f (eps2 d1 - eps4 d3) with d3 = (q2 - qm) - 3 d1, regrouped as
    // (L_f eps2 + 3 L_f eps4) d1 - L_f eps4 (q2 - qm); with Ls = 2 L_f the products below
    // are 2 b and 2 a3, so 2 d = a32 d1 - b2 e3 exactly as scaled
    const double Ls = w.Lam[dir][p] + w.Lam[dir][p + sd];
    const double b2 = Ls * eps4;
    const double a32 = fma(3.0, b2, Ls * eps2);
    for (int m = 0; m < 5; ++m) {
      const double* Q = q.q[m];
      const double d1 = Q[p + sd] - Q[p];
      const double e3 = Q[p + 2 * sd] - Q[p - sd];
      // twice the total face flux: (H_n + H_(n+1)) - 2 d_(n+1/2); the centred difference of H
      // and the dissipation difference then telescope into one difference of this flux
      const double hs = w.H[dir][m][p] + w.H[dir][m][p + sd];
      w.G[dir][m][p] = fma(-a32, d1, fma(b2, e3, hs));
    }
  }
}

// mode 0: stage update; mode 1: write RHS to rhs_flat (unpadded [5][N]).
template <int MODE>
__global__ void __launch_bounds__(kTPB) k_update(Dims d, GridDev g, Work64 w, State qin, State qn, State qout,
                                                 const Scalars* sc, double alpha, int want_res,
                                                 double* rhs_flat, double* res_sum) {
  Box b{0, 0, 0, d.ni, d.nj, d.nk};
  int i, j, k;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (box_coord(b, t, i, j, k)) {
    const long long p = pidx(d, i, j, k);
    const long long s[3] = {1, d.sj, d.sk};
    const bool adv = advanced(d, i, j);
    const double hV = 0.5 * g.invV[p];
    double R[5];                     // 2 V RHS; RHS = hV R
    for (int m = 0; m < 5; ++m) {
      // V RHS = sum_dir [(H+ - H-)/2 - (d+ - d-)] = (1/2) sum_dir (G(p) - G(p - s_dir)), with
      // G the doubled total face flux; the 1/(2V) goes into the update coefficient below
      const double* G0 = w.G[0][m];
      const double* G1 = w.G[1][m];
      const double* G2 = w.G[2][m];
      R[m] = ((G0[p] - G0[p - s[0]]) + (G1[p] - G1[p - s[1]])) + (G2[p] - G2[p - s[2]]);
    }
    if (MODE == 0) {
      const double adtV = alpha * sc->dt * hV;
      double qnew[5];
      for (int m = 0; m < 5; ++m) {
        qnew[m] = adv ? qn.q[m][p] - adtV * R[m] : qin.q[m][p];
        qout.q[m][p] = qnew[m];
      }
    } else {
      const long long N = (long long)d.ni * d.nj * d.nk;
      for (int m = 0; m < 5; ++m) rhs_flat[m * N + t] = adv ? R[m] * hV : 0.0;
    }
    if (adv) {
      const double r0 = R[0] * hV;
      r2 = r0 * r0;
    }
  }
  if (want_res) {
    // block sum of RHS_rho^2 -> one atomic per block
    __shared__ double red[kTPB / 32];
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
    __syncthreads();
    if (threadIdx.x < 32) {
      double x = threadIdx.x < kTPB / 32 ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (threadIdx.x == 0) atomicAdd(res_sum, x);
    }
  }
}

}  // namespace

cudaError_t nodal64(const Dims& d, const Consts& c, const GridDev& g, const Work64& w, const State& qin,
                    cudaStream_t st, double* rate_max) {
  const long long n0 = (long long)(d.ni + 2 * kG) * (d.nj + 2 * kG) * (d.nk + 2 * kG);
  k_nodal<<<blocks_for(n0, kTPB), kTPB, 0, st>>>(d, c, g, w, qin, rate_max);
  return cudaGetLastError();
}

cudaError_t viscous64(const Dims& d, const Consts& c, const GridDev& g, const Work64& w, const State& qin,
                      cudaStream_t st) {
  const long long n1 = (long long)(d.ni + 2) * (d.nj + 2) * (d.nk + 2);
  k_viscous<<<blocks_for(n1, kTPB), kTPB, 0, st>>>(d, c, g, w, qin);
  return cudaGetLastError();
}

cudaError_t faces64(const Dims& d, const Consts& c, const Work64& w, const State& qin, cudaStream_t st) {
  const long long nf = (long long)(d.ni + 1) * (d.nj + 1) * (d.nk + 1);
  k_faces<<<blocks_for(nf, kTPB), kTPB, 0, st>>>(d, c, w, qin);
  return cudaGetLastError();
}

cudaError_t update64(const Dims& d, const GridDev& g, const Work64& w, const State& qin, const State& qn,
                     const State& qout, const Scalars* sc, double alpha, int want_res, double* rhs_flat,
                     cudaStream_t st) {
  const long long nr = (long long)d.ni * d.nj * d.nk;
  double* res_sum = const_cast<double*>(&sc->res_sum);
  if (rhs_flat)
    k_update<1><<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, g, w, qin, qn, qout, sc, alpha, 0, rhs_flat, res_sum);
  else
    k_update<0><<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, g, w, qin, qn, qout, sc, alpha, want_res, nullptr,
                                                       res_sum);
  return cudaGetLastError();
}

}  // namespace jz
