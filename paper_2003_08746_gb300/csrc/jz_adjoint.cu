// Discrete adjoint of the FP64 Runge-Kutta stage, its boundary conditions and
// the observer functional (jz_adjoint_step).
//
// The forward stage (jz_stage64.cu) is: nodal pass -> viscous pass -> face
// pass -> RHS/update, then the boundary conditions (far field, entrance and
// exit, axis) and the ghost fill.  Its transpose runs backwards, each pass in
// "gather" form (every node or face sums the contributions it receives, so no
// two threads write the same address), except the transposed ghost map,
// which scatter-adds the adjoint of every ghost node onto the real node it
// copies.  Forward intermediates are recomputed from the stage input with
// the forward nodal and viscous kernels.  Non-smooth points take the same
// branch conventions as the forward code: max() gives its derivative to the
// first argument on ties, |x| and sqrt(x) at 0 have derivative 0, cbrt'(0)
// is 0, and the supersonic/subsonic and inflow/outflow switches take the
// branch the forward pass took.
#include "jz_adjgather.cuh"

namespace jz {
namespace {

constexpr int kTPB = 256;

__device__ __forceinline__ double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

__device__ __forceinline__ bool advanced(const Dims& d, int i, int j) {
  return d.topo != JZ_TOPO_JET || (i >= 1 && i <= d.ni - 2 && j >= 1 && j <= d.nj - 2);
}

// Reverse of u_i = m_i / rho, p = (gamma-1)(e - m.u/2) at one node: adds to qb.
__device__ __forceinline__ void prim_bar(const Consts& c, const double q[5], double ub[3], double pb, double qb[5]) {
  const double ir = rcp64(q[0]);
  const double u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  qb[4] += c.gm1 * pb;
  const double keb = -c.gm1 * pb;
  for (int a = 0; a < 3; ++a) {
    qb[1 + a] += 0.5 * keb * u[a];
    ub[a] += 0.5 * keb * q[1 + a];
  }
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    qb[1 + a] += ub[a] * ir;
    s += ub[a] * u[a];
  }
  qb[0] += -s * ir;
}

__device__ __forceinline__ void load5(const State& q, long long p, double v[5]) {
  for (int m = 0; m < 5; ++m) v[m] = q.q[m][p];
}

// ---- update: Qn_bar += lam, acc = -alpha dt (1/V) lam on advanced nodes ----------
__global__ void k_adj_update(Dims d, GridDev g, Adj64 a, double adt) {
  Box b{0, 0, 0, d.ni, d.nj, d.nk};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const bool adv = advanced(d, i, j);
  const double iV = g.invV[p];
  for (int m = 0; m < 5; ++m) {
    const double l = a.lam[m][p];
    if (adv) a.qnbar[m][p] += l;
    a.acc[m][p] = adv ? -adt * l * iV : 0.0;
  }
}

// ---- dissipation faces (FP64 solvers; pair solvers: jz_adjointdf.cu) ----------------
__global__ void k_adj_faces(Dims d, Consts c, Work64 w, State q, Adj64 a) {
  Box b{-1, -1, -1, d.ni + 1, d.nj + 1, d.nk + 1};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const long long s[3] = {1, d.sj, d.sk};
  for (int dir = 0; dir < 3; ++dir) {
    const long long sd = s[dir];
    const double nu0 = w.nu[dir][p], nu1 = w.nu[dir][p + sd];
    const bool first = nu0 >= nu1;
    const double eps2 = c.kappa2 * (first ? nu0 : nu1);
    const double k4 = c.kappa4 - eps2;
    const double eps4 = k4 > 0.0 ? k4 : 0.0;
    const double Lf = 0.5 * (w.Lam[dir][p] + w.Lam[dir][p + sd]);
    double lf = 0.0, e2b = 0.0, e4b = 0.0;
    for (int m = 0; m < 5; ++m) {
      const double* Q = q.q[m];
      const double q0 = Q[p], q1 = Q[p + sd], q2 = Q[p + 2 * sd], qm = Q[p - sd];
      const double d1 = q1 - q0;
      const double d3 = q2 - 3.0 * q1 + 3.0 * q0 - qm;
      const double Db = a.acc[m][p + sd] - a.acc[m][p];
      lf += Db * (eps2 * d1 - eps4 * d3);
      e2b += Db * Lf * d1;
      e4b += -Db * Lf * d3;
    }
    // the face adjoints of d1 and d3 are Db Lf eps2 and -Db Lf eps4: the nodal gather forms them
    // from these two coefficients and the differences of acc it reads anyway
    a.ca2[dir][p] = Lf * eps2;
    a.ca4[dir][p] = Lf * eps4;
    if (k4 > 0.0) e2b += -e4b;
    const double nub = c.kappa2 * e2b;
    a.nb0[dir][p] = first ? nub : 0.0;
    a.nb1[dir][p] = first ? 0.0 : nub;
    a.lfh[dir][p] = 0.5 * lf;
  }
}

// ---- viscous pass and pressure sensor (FP64 solvers; pair solvers: jz_adjointdf.cu) --
__global__ void k_adj_visc(Dims d, Consts c, GridDev g, Work64 w, State q, Adj64 a) {
  Box b{-1, -1, -1, d.ni + 2, d.nj + 2, d.nk + 2};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const long long s[3] = {1, d.sj, d.sk};
  // adjoint of H^dir (components 1..4 carry the viscous flux)
  double Hb[3][4];
  for (int dir = 0; dir < 3; ++dir)
    for (int m = 0; m < 4; ++m)
      Hb[dir][m] = 0.5 * (a.acc[m + 1][p - s[dir]] - a.acc[m + 1][p + s[dir]]);
  // forward viscous quantities
  const double* f[4] = {w.u, w.v, w.w, w.T};
  double S[3][3];
  for (int dir = 0; dir < 3; ++dir)
    for (int cc = 0; cc < 3; ++cc) S[dir][cc] = g.S[3 * dir + cc][p];
  const double iV = g.invV[p];
  double L[4][3];
  for (int n = 0; n < 4; ++n) {
    double dd[3];
    for (int dir = 0; dir < 3; ++dir) dd[dir] = 0.5 * (f[n][p + s[dir]] - f[n][p - s[dir]]);
    for (int jj = 0; jj < 3; ++jj) L[n][jj] = iV * (S[0][jj] * dd[0] + S[1][jj] * dd[1] + S[2][jj] * dd[2]);
  }
  double Sij[3][3];
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) Sij[x][y] = 0.5 * (L[x][y] + L[y][x]);
  const double div = Sij[0][0] + Sij[1][1] + Sij[2][2];
  double SS = 0.0;
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) SS = SS + Sij[x][y] * Sij[x][y];
  const double Smod = sqrt64(2.0 * SS);
  const double mu = w.mu[p];
  const double csd = c.C_s * g.Delta[p];
  const double rho = q.q[0][p];
  const double mu_sgs = rho * (csd * csd) * Smod;
  const double mu_eff = mu + mu_sgs;
  const double k_eff = mu * c.k_lam + mu_sgs * c.k_sgs;
  const double d3 = div * (1.0 / 3.0);
  double tau[3][3];
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) tau[x][y] = 2.0 * mu_eff * (Sij[x][y] - (x == y ? d3 : 0.0));
  const double vel[3] = {w.u[p], w.v[p], w.w[p]};
  // reverse: F^dir_m = S^dir_j F_j,m ; H = E - F
  double Fb[3][4];
  for (int jj = 0; jj < 3; ++jj)
    for (int m = 0; m < 4; ++m) Fb[jj][m] = -(S[0][jj] * Hb[0][m] + S[1][jj] * Hb[1][m] + S[2][jj] * Hb[2][m]);
  double taub[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double ubd[3] = {0, 0, 0}, keb = 0.0, L3b[3] = {0, 0, 0};
  for (int jj = 0; jj < 3; ++jj) {
    for (int x = 0; x < 3; ++x) taub[x][jj] += Fb[jj][x];
    const double e = Fb[jj][3];
    for (int x = 0; x < 3; ++x) {
      ubd[x] += e * tau[x][jj];
      taub[x][jj] += e * vel[x];
    }
    keb += e * L[3][jj];
    L3b[jj] += e * k_eff;
  }
  double mueb = 0.0, Sijb[3][3], divb = 0.0;
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) {
      mueb += taub[x][y] * 2.0 * (Sij[x][y] - (x == y ? d3 : 0.0));
      Sijb[x][y] = 2.0 * mu_eff * taub[x][y];
    }
  for (int x = 0; x < 3; ++x) divb += -(mu_eff * (2.0 / 3.0)) * taub[x][x];
  for (int x = 0; x < 3; ++x) Sijb[x][x] += divb;
  const double mub = keb * c.k_lam + mueb;
  const double musb = keb * c.k_sgs + mueb;
  const double rhob = musb * (csd * csd) * Smod;
  const double Smodb = musb * rho * (csd * csd);
  const double SSb = Smod > 0.0 ? Smodb * rcp64(Smod) : 0.0;
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) Sijb[x][y] += 2.0 * Sij[x][y] * SSb;
  double Lb[4][3];
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) Lb[x][y] = 0.5 * (Sijb[x][y] + Sijb[y][x]);
  for (int y = 0; y < 3; ++y) Lb[3][y] = L3b[y];
  for (int n = 0; n < 4; ++n)
    for (int dir = 0; dir < 3; ++dir)
      a.G[n][dir][p] = iV * (S[dir][0] * Lb[n][0] + S[dir][1] * Lb[n][1] + S[dir][2] * Lb[n][2]);
  for (int x = 0; x < 3; ++x) a.ubd[x][p] = ubd[x];
  a.mub[p] = mub;
  a.rhob[p] = rhob;
  // pressure sensor nu = |N|/Dn
  const double pc = w.p[p];
  for (int dir = 0; dir < 3; ++dir) {
    const double nub = a.nb0[dir][p] + a.nb1[dir][p - s[dir]];
    const double pp = w.p[p + s[dir]], pm = w.p[p - s[dir]];
    const double N = pp - 2.0 * pc + pm, Dn = pp + 2.0 * pc + pm;
    const double iD = rcp64(Dn);
    const double nu = fabs(N) * iD;
    a.cpm[dir][p] = nub * (sgn(N) - nu) * iD;
    a.c0[dir][p] = nub * (-2.0 * sgn(N) - 2.0 * nu) * iD;
  }
}

// ---- nodal pass: gathers, then the reverse of primitives/fluxes/spectral radii (FP64) --
// 128-thread blocks, three per SM: the pass needs ~170 registers, and three small blocks
// keep more warps resident than one 256-thread block (4% faster gradient).
constexpr int kTPBN = 128;
__global__ void __launch_bounds__(kTPBN, 3) k_adj_nodal(Dims d, Consts c, GridDev g, Work64 w, State q, Adj64 a) {
  Box b{-kG, -kG, -kG, d.ni + 2 * kG, d.nj + 2 * kG, d.nk + 2 * kG};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  NodalGathers G;
  nodal_gathers(d, a, i, j, k, G);
  double* fb = G.fb;
  double pb = G.pb;
  double (*Eb)[5] = G.Eb;
  double* Lamb = G.Lamb;
  double* qb = G.qb;
  const double mub = G.mub;
  // forward nodal quantities
  double Q[5];
  load5(q, p, Q);
  const double rho = Q[0];
  const double ir = rcp64(rho);
  const double u[3] = {Q[1] * ir, Q[2] * ir, Q[3] * ir};
  const double pr = c.gm1 * (Q[4] - 0.5 * (Q[1] * u[0] + Q[2] * u[1] + Q[3] * u[2]));
  const double T = c.gamma * pr * ir;
  const double aa = sqrt64(T);
  const double iTS = rcp64(T + c.S_hat);
  const double mu = c.mu_ref * (T * aa) * c.sut_num * iTS;
  double Sv[3][3], Smag[3], U[3], lam[3];
  for (int dir = 0; dir < 3; ++dir) {
    for (int cc = 0; cc < 3; ++cc) Sv[dir][cc] = g.S[3 * dir + cc][p];
    Smag[dir] = g.Smag[dir][p];
    U[dir] = Sv[dir][0] * u[0] + Sv[dir][1] * u[1] + Sv[dir][2] * u[2];
    lam[dir] = fabs(U[dir]) + aa * Smag[dir];
  }
  // anisotropic scaling Lambda_d = lam_d + lo_d (hi_e + hi_f)
  double lamb[3] = {Lamb[0], Lamb[1], Lamb[2]};
  {
    double lo[3], hi[3], dlo[3], dhi[3];
    for (int dd = 0; dd < 3; ++dd) {
      if (c.sigma_is_two_thirds) {
        double t, t2;
        cbrt_pair64(lam[dd], t, t2);                        // lam^(1/3), lam^(2/3)
        lo[dd] = t;
        hi[dd] = t2;
        dlo[dd] = t != 0.0 ? rcp64(3.0 * t2) : 0.0;         // d t / d lam
        dhi[dd] = 2.0 * t * dlo[dd];                        // d t^2 / d lam
      } else {
        const bool pos = lam[dd] > 0.0;
        lo[dd] = pos ? pow(lam[dd], 1.0 - c.sigma) : 0.0;
        hi[dd] = pos ? pow(lam[dd], c.sigma) : 0.0;
        dlo[dd] = pos ? (1.0 - c.sigma) * lo[dd] / lam[dd] : 0.0;
        dhi[dd] = pos ? c.sigma * hi[dd] / lam[dd] : 0.0;
      }
    }
    double lob[3] = {0, 0, 0}, hib[3] = {0, 0, 0};
    const int e1[3] = {1, 0, 0}, e2[3] = {2, 2, 1};
    for (int dd = 0; dd < 3; ++dd) {
      lob[dd] += Lamb[dd] * (hi[e1[dd]] + hi[e2[dd]]);
      hib[e1[dd]] += Lamb[dd] * lo[dd];
      hib[e2[dd]] += Lamb[dd] * lo[dd];
    }
    for (int dd = 0; dd < 3; ++dd) lamb[dd] += lob[dd] * dlo[dd] + hib[dd] * dhi[dd];
  }
  double Ub[3], ab = 0.0;
  double ub[3] = {fb[0], fb[1], fb[2]};
  double Tb = fb[3];
  for (int dir = 0; dir < 3; ++dir) {
    Ub[dir] = lamb[dir] * sgn(U[dir]);
    ab += lamb[dir] * Smag[dir];
    // E = [rho U, m_i U + p S_i, (e + p) U]
    qb[0] += Eb[dir][0] * U[dir];
    Ub[dir] += Eb[dir][0] * rho;
    for (int x = 0; x < 3; ++x) {
      qb[1 + x] += Eb[dir][1 + x] * U[dir];
      Ub[dir] += Eb[dir][1 + x] * Q[1 + x];
      pb += Eb[dir][1 + x] * Sv[dir][x];
    }
    qb[4] += Eb[dir][4] * U[dir];
    pb += Eb[dir][4] * U[dir];
    Ub[dir] += Eb[dir][4] * (Q[4] + pr);
    for (int x = 0; x < 3; ++x) ub[x] += Ub[dir] * Sv[dir][x];
  }
  // Sutherland mu(T): d mu / dT = mu (1.5/T - 1/(T + S))
  Tb += mub * mu * (1.5 * rcp64(T) - iTS);
  Tb += ab * 0.5 * rcp64(aa);
  pb += Tb * c.gamma * ir;
  qb[0] += -Tb * T * ir;
  prim_bar(c, Q, ub, pb, qb);
  for (int m = 0; m < 5; ++m) a.lam[m][p] = qb[m];
}

// ---- transposed ghost map: ghost adjoint added onto its source node --------------
__device__ __forceinline__ bool ghost_coord_adj(const Dims& d, long long t, int& i, int& j, int& k) {
  const long long ei = d.ni + 2 * kG, ej = d.nj + 2 * kG;
  const long long nA = 4 * ei * ej, nB = 4 * ei * d.nk, nC = 4LL * d.nj * d.nk;
  if (t < nA) {
    i = (int)(t % ei) - kG;
    const long long r = t / ei;
    j = (int)(r % ej) - kG;
    const int s = (int)(r / ej);
    k = s < 2 ? s - 2 : d.nk + s - 2;
    return true;
  }
  t -= nA;
  if (t < nB) {
    i = (int)(t % ei) - kG;
    const long long r = t / ei;
    const int s = (int)(r % 4);
    k = (int)(r / 4);
    j = s < 2 ? s - 2 : d.nj + s - 2;
    return true;
  }
  t -= nB;
  if (t < nC) {
    const int s = (int)(t % 4);
    const long long r = t / 4;
    j = (int)(r % d.nj);
    k = (int)(r / d.nj);
    i = s < 2 ? s - 2 : d.ni + s - 2;
    return true;
  }
  return false;
}

__global__ void k_adj_ghost(Dims d, Adj64 a) {
  int i, j, k;
  if (!ghost_coord_adj(d, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  int si, sj, sk;
  ghost_source(d, i, j, k, si, sj, sk);
  const long long p = pidx(d, i, j, k), q = pidx(d, si, sj, sk);
  for (int m = 0; m < 5; ++m) {
    const double v = a.lam[m][p];
    if (v != 0.0) atomicAdd(&a.lam[m][q], v);
  }
}

__global__ void k_adj_addqn(Dims d, Adj64 a) {
  Box b{0, 0, 0, d.ni, d.nj, d.nk};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  for (int m = 0; m < 5; ++m) {
    a.lam[m][p] += a.qnbar[m][p];
    a.qnbar[m][p] = 0.0;
  }
}

// ---- boundary-condition adjoints (reverse order: axis, entrance/exit, far field) ----
__global__ void k_adj_axis(Dims d, Adj64 a) {
  const int i = blockIdx.x;
  double s[5] = {0, 0, 0, 0, 0};
  for (int k = threadIdx.x; k < d.nk; k += blockDim.x) {
    const long long p = pidx(d, i, 0, k);
    for (int m = 0; m < 5; ++m) s[m] += a.lam[m][p];
  }
  __shared__ double red[5][4];
  for (int m = 0; m < 5; ++m) {
    double x = s[m];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[m][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  double add[5];
  for (int m = 0; m < 5; ++m) add[m] = (red[m][0] + red[m][1] + red[m][2] + red[m][3]) / d.nk;
  for (int k = threadIdx.x; k < d.nk; k += blockDim.x) {
    const long long p0 = pidx(d, i, 0, k), p1 = pidx(d, i, 1, k);
    for (int m = 0; m < 5; ++m) {
      a.lam[m][p1] += add[m];
      a.lam[m][p0] = 0.0;
    }
  }
}

__global__ void k_adj_inout(Dims d, Consts c, Inflow in, State q, Adj64 a, double ts) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nj1 = d.nj - 1;
  const long long nface = (long long)nj1 * d.nk;
  const long long plane = (long long)d.nk * d.nj;
  double g0 = 0.0;                 // d J / d u_target (times U_j) at this entrance node
  long long tab = 0;
  // temporal factors sin(omega_f t + psi_mf), uniform over the entrance: once per block
  __shared__ double sn[kNF];
  if (threadIdx.x < kNF) sn[threadIdx.x] = sin(in.omega[threadIdx.x % JZ_N_FREQ] * ts + in.psi[threadIdx.x]);
  __syncthreads();
  if (t < 2 * nface) {
    const bool exit_plane = t >= nface;
    const long long tt = exit_plane ? t - nface : t;
    const int j = 1 + (int)(tt % nj1), k = (int)(tt / nj1);
    if (!exit_plane) {
      const long long pb = pidx(d, 0, j, k), p1 = pidx(d, 1, j, k);
      tab = (long long)k * d.nj + j;
      double f = 0.0;
      for (int mf = 0; mf < kNF; ++mf)
        f = f + in.amp[mf] * in.Gf[mf * plane + tab] * sn[mf];
      const double ut = in.u0[tab] + c.jet_mach * f;
      double Q1[5];
      load5(q, p1, Q1);
      double lb[5];
      for (int m = 0; m < 5; ++m) lb[m] = a.lam[m][pb];
      double utb;
      const bool sup = ut >= 1.0;
      if (sup) {
        utb = lb[1] + lb[4] * ut;
      } else {
        const double rho1 = Q1[0];
        const double u1 = Q1[1] / rho1;
        const double pr1 = c.gm1 * (Q1[4] - 0.5 * (Q1[1] * Q1[1] + Q1[2] * Q1[2] + Q1[3] * Q1[3]) / rho1);
        const double a1 = sqrt(c.gamma * pr1 / rho1);
        const double Rm = u1 - 2.0 * a1 / c.gm1, Rp = ut + 2.0 * 1.0 / c.gm1;
        const double ub = 0.5 * (Rp + Rm), ab = 0.25 * c.gm1 * (Rp - Rm);
        const double rs = pow(ab * ab / (c.gamma * c.p_inf), 1.0 / c.gm1);
        const double rhob = lb[0] + lb[1] * ub + 0.5 * lb[4] * ub * ub;
        const double ubb = lb[1] * rs + lb[4] * rs * ub;
        const double pbb = lb[4] / c.gm1;
        double rsb = rhob + pbb * ab * ab / c.gamma;
        double abb = pbb * 2.0 * rs * ab / c.gamma;
        abb += rsb * 2.0 * rs / (c.gm1 * ab);
        const double Rpb = 0.5 * ubb + 0.25 * c.gm1 * abb;
        const double Rmb = 0.5 * ubb - 0.25 * c.gm1 * abb;
        utb = Rpb;
        double u1b[3] = {Rmb, 0.0, 0.0};
        const double a1b = -2.0 * Rmb / c.gm1;
        const double p1b = a1b * c.gamma / (2.0 * a1 * rho1);
        double q1b[5] = {-a1b * c.gamma * pr1 / (2.0 * a1 * rho1 * rho1), 0, 0, 0, 0};
        prim_bar(c, Q1, u1b, p1b, q1b);
        for (int m = 0; m < 5; ++m) a.lam[m][p1] += q1b[m];
      }
      g0 = utb * c.jet_mach;
      for (int m = 0; m < 5; ++m) a.lam[m][pb] = 0.0;
    } else {
      const long long pi = pidx(d, d.ni - 2, j, k), pb = pidx(d, d.ni - 1, j, k);
      double Qi[5];
      load5(q, pi, Qi);
      const double rho_i = Qi[0];
      const double u[3] = {Qi[1] / rho_i, Qi[2] / rho_i, Qi[3] / rho_i};
      const double p_i = c.gm1 * (Qi[4] - 0.5 * (Qi[1] * u[0] + Qi[2] * u[1] + Qi[3] * u[2]));
      const double rho = c.p_inf / (c.gm1 * (p_i / (c.gm1 * rho_i)));
      double lb[5];
      for (int m = 0; m < 5; ++m) lb[m] = a.lam[m][pb];
      const double rhob = lb[0] + lb[1] * u[0] + lb[2] * u[1] + lb[3] * u[2] +
                          0.5 * lb[4] * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      double ub[3];
      for (int x = 0; x < 3; ++x) ub[x] = lb[1 + x] * rho + lb[4] * rho * u[x];
      double qb[5] = {rhob * rho / rho_i, 0, 0, 0, 0};
      const double pib = -rhob * rho / p_i;
      prim_bar(c, Qi, ub, pib, qb);
      for (int m = 0; m < 5; ++m) {
        a.lam[m][pi] += qb[m];
        a.lam[m][pb] = 0.0;
      }
    }
  }
  // dJ/dA_mf = sum over the entrance of g0 G_mf sin(omega_f t + psi_mf): block sums,
  // one atomic per parameter per block
  __shared__ double red[kNF][kTPB / 32];
  for (int f = 0; f < kNF; ++f) {
    double x = g0 != 0.0 ? g0 * in.Gf[f * plane + tab] * sn[f] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[f][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < kNF) {
    double x = 0.0;
    for (int w = 0; w < kTPB / 32; ++w) x += red[threadIdx.x][w];
    if (x != 0.0) atomicAdd(&a.abar[threadIdx.x], x);
  }
}

__global__ void k_adj_farfield(Dims d, Consts c, GridDev g, State q, Adj64 a) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int ni2 = d.ni - 2;
  if (t >= (long long)ni2 * d.nk) return;
  const int i = 1 + (int)(t % ni2), k = (int)(t / ni2);
  const int jb = d.nj - 1;
  const long long pb = pidx(d, i, jb, k), pi = pidx(d, i, jb - 1, k);
  const long long nsurf = (long long)d.nk * d.ni, isurf = (long long)k * d.ni + i;
  const double sx = g.Sb[isurf], sy = g.Sb[nsurf + isurf], sz = g.Sb[2 * nsurf + isurf];
  const double nm = sqrt(sx * sx + sy * sy + sz * sz);
  const double n[3] = {sx / nm, sy / nm, sz / nm};
  double Qi[5];
  load5(q, pi, Qi);
  const double rho_i = Qi[0];
  const double ui[3] = {Qi[1] / rho_i, Qi[2] / rho_i, Qi[3] / rho_i};
  const double p_i = c.gm1 * (Qi[4] - 0.5 * (Qi[1] * ui[0] + Qi[2] * ui[1] + Qi[3] * ui[2]));
  const double a_i = sqrt(c.gamma * p_i / rho_i);
  const double un_i = ui[0] * n[0] + ui[1] * n[1] + ui[2] * n[2];
  const double Rp = un_i + 2.0 * a_i / c.gm1, Rm = -2.0 / c.gm1;
  const double un = 0.5 * (Rp + Rm), ab = 0.25 * c.gm1 * (Rp - Rm);
  const bool out = un > 0.0;
  double ut[3];
  for (int x = 0; x < 3; ++x) ut[x] = out ? ui[x] - un_i * n[x] : 0.0;
  const double s = out ? p_i / pow(rho_i, c.gamma) : c.p_inf;
  const double rho = pow(ab * ab / (c.gamma * s), 1.0 / c.gm1);
  double ubv[3];
  for (int x = 0; x < 3; ++x) ubv[x] = ut[x] + un * n[x];
  double lb[5];
  for (int m = 0; m < 5; ++m) lb[m] = a.lam[m][pb];
  double rhob = lb[0] + 0.5 * lb[4] * (ubv[0] * ubv[0] + ubv[1] * ubv[1] + ubv[2] * ubv[2]);
  double ubb[3];
  for (int x = 0; x < 3; ++x) {
    rhob += lb[1 + x] * ubv[x];
    ubb[x] = lb[1 + x] * rho + lb[4] * rho * ubv[x];
  }
  const double pbb = lb[4] / c.gm1;
  rhob += pbb * ab * ab / c.gamma;
  double abb = pbb * 2.0 * rho * ab / c.gamma;
  abb += rhob * 2.0 * rho / (c.gm1 * ab);
  const double sb = -rhob * rho / (c.gm1 * s);
  double unb = 0.0;
  for (int x = 0; x < 3; ++x) unb += ubb[x] * n[x];
  const double Rpb = 0.5 * unb + 0.25 * c.gm1 * abb;
  double un_ib = Rpb;
  const double a_ib = 2.0 * Rpb / c.gm1;
  double uib[3] = {0, 0, 0};
  double p_ib = 0.0;
  double qb[5] = {0, 0, 0, 0, 0};
  if (out) {
    double tn = 0.0;
    for (int x = 0; x < 3; ++x) {
      uib[x] += ubb[x];
      tn += ubb[x] * n[x];
    }
    un_ib += -tn;
    const double rg = pow(rho_i, -c.gamma);
    p_ib += sb * rg;
    qb[0] += -c.gamma * sb * s / rho_i;
  }
  for (int x = 0; x < 3; ++x) uib[x] += un_ib * n[x];
  p_ib += a_ib * c.gamma / (2.0 * a_i * rho_i);
  qb[0] += -a_ib * c.gamma * p_i / (2.0 * a_i * rho_i * rho_i);
  prim_bar(c, Qi, uib, p_ib, qb);
  for (int m = 0; m < 5; ++m) {
    a.lam[m][pi] += qb[m];
    a.lam[m][pb] = 0.0;
  }
}

// ---- observer functional: value and adjoint at one time level --------------------
__global__ void k_observer(Dims d, Consts c, State q, const double* w, int j0, double beta, double dt, Adj64 a,
                           int want_grad) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double val = 0.0;
  if (t < (long long)d.ni * d.nk) {
    const int i = (int)(t % d.ni), k = (int)(t / d.ni);
    const long long p0 = pidx(d, i, j0, k), p1 = pidx(d, i, j0 + 1, k);
    double Q0[5], Q1[5];
    load5(q, p0, Q0);
    load5(q, p1, Q1);
    auto pres = [&](const double* Q) {
      return c.gm1 * (Q[4] - 0.5 * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]) / Q[0]);
    };
    const double pt = (1.0 - beta) * pres(Q0) + beta * pres(Q1);
    const double dp = pt - c.p_inf;
    val = dt * w[i] * dp * dp;
    if (want_grad) {
      const double gsc = 2.0 * dt * w[i] * dp;
      const double wt[2] = {1.0 - beta, beta};
      const long long pp[2] = {p0, p1};
      const double* QQ[2] = {Q0, Q1};
      for (int s = 0; s < 2; ++s) {
        const double pb = gsc * wt[s];
        const double* Q = QQ[s];
        const double m2 = Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3];
        a.lam[0][pp[s]] += pb * c.gm1 * 0.5 * m2 / (Q[0] * Q[0]);
        for (int x = 0; x < 3; ++x) a.lam[1 + x][pp[s]] += -pb * c.gm1 * Q[1 + x] / Q[0];
        a.lam[4][pp[s]] += pb * c.gm1;
      }
    }
  }
  __shared__ double red[kTPB / 32];
  for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int w2 = 0; w2 < kTPB / 32; ++w2) x += red[w2];
    if (!want_grad) atomicAdd(a.J, x);
  }
}

__global__ void k_set_time(Scalars* sc, double t, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->t = t;
    sc->dt = dt;
  }
}

}  // namespace

cudaError_t adj_update(const Dims& d, const GridDev& g, const Adj64& a, double adt, cudaStream_t st) {
  const long long nr = (long long)d.ni * d.nj * d.nk;
  k_adj_update<<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, g, a, adt);
  return cudaGetLastError();
}

cudaError_t adj_stage(const Dims& d, const Consts& c, const GridDev& g, const Work64& w, const State& q,
                      const Adj64& a, const DFMetrics* mdf, const QDF* qdf, cudaStream_t st) {
  const bool pair = mdf && qdf;
  const long long n0 = (long long)(d.ni + 2 * kG) * (d.nj + 2 * kG) * (d.nk + 2 * kG);
  const long long n1 = (long long)(d.ni + 2) * (d.nj + 2) * (d.nk + 2);
  const long long nf = (long long)(d.ni + 1) * (d.nj + 1) * (d.nk + 1);
  if (pair) {
    cudaError_t e = adj_faces_df(d, c, w, *qdf, a, st);
    if (e == cudaSuccess) e = adj_visc_df(d, c, *mdf, w, *qdf, a, st);
    if (e == cudaSuccess) e = adj_nodal_df(d, c, *mdf, *qdf, a, st);
    if (e != cudaSuccess) return e;
  } else {
    k_adj_faces<<<blocks_for(nf, kTPB), kTPB, 0, st>>>(d, c, w, q, a);
    k_adj_visc<<<blocks_for(n1, kTPB), kTPB, 0, st>>>(d, c, g, w, q, a);
    k_adj_nodal<<<blocks_for(n0, kTPBN), kTPBN, 0, st>>>(d, c, g, w, q, a);
  }
  const long long ei = d.ni + 2 * kG, ej = d.nj + 2 * kG;
  const long long ng = 4 * ei * ej + 4 * ei * d.nk + 4LL * d.nj * d.nk;
  k_adj_ghost<<<blocks_for(ng, kTPB), kTPB, 0, st>>>(d, a);
  return cudaGetLastError();
}

cudaError_t adj_add_qn(const Dims& d, const Adj64& a, cudaStream_t st) {
  const long long nr = (long long)d.ni * d.nj * d.nk;
  k_adj_addqn<<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, a);
  return cudaGetLastError();
}

cudaError_t adj_bcs(const Dims& d, const Consts& c, const GridDev& g, const Inflow& in, const State& q,
                    const Adj64& a, double ts, cudaStream_t st) {
  if (d.topo != JZ_TOPO_JET) return cudaSuccess;
  k_adj_axis<<<d.ni, 128, 0, st>>>(d, a);
  const long long nio = 2LL * (d.nj - 1) * d.nk;
  k_adj_inout<<<blocks_for(nio, kTPB), kTPB, 0, st>>>(d, c, in, q, a, ts);
  const long long nf = (long long)(d.ni - 2) * d.nk;
  k_adj_farfield<<<blocks_for(nf, kTPB), kTPB, 0, st>>>(d, c, g, q, a);
  return cudaGetLastError();
}

cudaError_t observer(const Dims& d, const Consts& c, const State& q, const double* w, int j0, double beta,
                     double dt, const Adj64& a, int want_grad, cudaStream_t st) {
  const long long n = (long long)d.ni * d.nk;
  k_observer<<<blocks_for(n, kTPB), kTPB, 0, st>>>(d, c, q, w, j0, beta, dt, a, want_grad);
  return cudaGetLastError();
}

cudaError_t set_time(Scalars* sc, double t, double dt, cudaStream_t st) {
  k_set_time<<<1, 32, 0, st>>>(sc, t, dt);
  return cudaGetLastError();
}

}  // namespace jz
