// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/jz.h"

namespace jz {

constexpr int kG = 2;            // ghost layers per side (two-layer ghosts)
constexpr int kNF = JZ_N_MODES * JZ_N_FREQ;

// Padded box geometry.  Real node (i, j, k), -2 <= i <= ni + 1, sits at
// element ((k + 2) * Pj + (j + 2)) * Pi + (i + 2).  Pi is rounded up to a
// multiple of 4 elements so that every row starts 32-byte aligned; the
// columns past i = ni + 1 are never read by the stencil.
struct Dims {
  int ni, nj, nk;
  int Pi, Pj, Pk;
  long long Np;                  // padded elements per field
  long long sj, sk;              // element strides of j and k
  int topo;
};

__host__ __device__ inline long long pidx(const Dims& d, int i, int j, int k) {
  return ((long long)(k + kG) * d.Pj + (j + kG)) * d.Pi + (i + kG);
}

inline Dims make_dims(int ni, int nj, int nk, int topo) {
  Dims d;
  d.ni = ni; d.nj = nj; d.nk = nk; d.topo = topo;
  d.Pi = ((ni + 2 * kG) + 3) / 4 * 4;
  d.Pj = nj + 2 * kG;
  d.Pk = nk + 2 * kG;
  d.sj = d.Pi;
  d.sk = (long long)d.Pi * d.Pj;
  d.Np = d.sk * d.Pk;
  return d;
}

// FP64 reciprocal, square root and cube root with fewer FP64-pipe instructions
// than IEEE division and the library routines; the FP64 form is bound by that
// pipe (about 1/64 of an SM sub-partition's issue rate), while integer and
// FP32 work issues almost for free beside it.  All three are accurate to about
// one unit in the last place (checked against 1.0/x, sqrt(x) and cbrt(x) by
// jz_check_math), far inside the form's 1e-12 parity.
//
// The refinements are the third-order (Householder) iterations for a root:
// with a seed y of r = x^(1/n) or of 1/r and the residual e = 1 - (seed
// relation), the exact correction factor (1 - e)^(-1/n) is expanded to its e^2
// term, so a seed good to ~2^-22 lands below 2^-60 before the final rounding.
//
// rcp64: for normal, finite x != 0.  Seed: the hardware approximation
// rcp.approx.ftz.f64 (about 2^-22 relative); with e = 1 - x r,
//   1/x = r / (1 - e) ~ r (1 + e + e^2)         (three FMAs).
__device__ __forceinline__ double rcp64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// FP64 <-> FP32 by integer operations on the IEEE fields (mantissa truncated;
// exponent re-biased by 1023 - 127 = 896), valid for 2^-100 <= |x| < 2^101,
// so that the seeds below stay off the FP64 pipe.
__device__ __forceinline__ float seed_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  return __uint_as_float(((hi - (896u << 20)) << 3) | (lo >> 29));
}
__device__ __forceinline__ double seed_f64(float f) {
  const unsigned b = __float_as_uint(f);
  return __hiloint2double((int)((b >> 3) + (896u << 20)), (int)(b << 29));
}
// true when 2^-100 <= x < 2^101 (x >= 0 assumed; also false for 0, Inf, NaN)
__device__ __forceinline__ bool seed_range(double x) {
  return (unsigned)__double2hiint(x) - ((1023u - 100u) << 20) < (201u << 20);
}

// sqrt64: sqrt(x) for x >= 0.  Seed z ~ x^(-1/2) from the FP32 MUFU
// rsqrt.approx; with e = 1 - x z^2,
//   sqrt(x) = x z (1 - e)^(-1/2) ~ w + w e (1/2 + 3e/8),   w = x z.
// Arguments outside [2^-100, 2^101) (0 among them) use the library sqrt.
__device__ __forceinline__ double sqrt64(double x) {
  if (!seed_range(x)) return sqrt(x);
  float zf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(zf) : "f"(seed_f32(x)));
  const double z = seed_f64(zf);
  const double e = fma(-x, z * z, 1.0);
  const double w = x * z;
  return fma(w, e * fma(0.375, e, 0.5), w);
}

// cbrt_pair64: c1 = x^(1/3) and c2 = x^(2/3) for x >= 0.  Seed z ~ x^(-1/3)
// = 2^(-log2(x)/3) in FP32 (MUFU lg2 and ex2); with e = 1 - x z^3,
//   x^(-1/3) = z (1 - e)^(-1/3) ~ z (1 + u),   u = e (1/3 + 2e/9),
//   x^(2/3) = x z (1 + u),   x^(1/3) = x^(2/3) z (1 + u).
// Arguments outside [2^-100, 2^101) (0 among them) use the library cube root.
__device__ __forceinline__ void cbrt_pair64(double x, double& c1, double& c2) {
  if (!seed_range(x)) {
    c1 = cbrt(x);
    c2 = c1 * c1;
    return;
  }
  float l, zf;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(seed_f32(x)));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(zf) : "f"(l * (-1.0f / 3.0f)));
  const double z = seed_f64(zf);
  const double w = x * z;                       // ~ x^(2/3)
  const double e = fma(-w, z * z, 1.0);
  const double u = e * fma(2.0 / 9.0, e, 1.0 / 3.0);
  c2 = fma(w, u, w);
  c1 = c2 * fma(z, u, z);
}

__device__ __forceinline__ double cbrt64(double x) {
  double c1, c2;
  cbrt_pair64(x, c1, c2);
  return c1;
}

// Grid arrays on the device (padded, ghost-filled).
struct GridDev {
  double* xyz[3];
  double* S[9];       // S^xi_{x,y,z}, S^eta_{x,y,z}, S^zeta_{x,y,z}
  double* V;          // cell volume 1/J
  double* invV;       // 1/V (0 where V = 0, i.e. on the jet axis)
  double* Smag[3];    // |S^dir|
  double* Delta;      // filter width V^(1/3)
  // surface copies kept by every grid (also compact ones)
  double* Sb;         // far-field normals S^eta at j = nj-1: [3][nk][ni]
  double* Xin;        // entrance-plane coordinates y, z at i = 0: [2][nk][nj]
  // compact grids (jz_grid_compact): the FP64 arrays above except Sb and Xin are
  // released and the metrics are kept in FP32 only
  int compact;
  const float* Mf;    // compact grids: the FP32 metric records (kMF floats per padded node)
};

// FP32 metric record of one padded node (the FP32-flux form): S^xi, S^eta, S^zeta (9),
// V, 1/V (0 where V = 0), V^(1/3); 48 bytes, read as three 16-byte vectors.
constexpr int kMF = 12;
constexpr int MF_V = 9, MF_IV = 10, MF_D = 11;

// Derived constants of the non-dimensional formulation, by value.
struct Consts {
  double gamma, gm1, Cp;
  double mu_ref, S_hat, sut_num;   // sut_num = 1 + S_hat
  double k_lam, k_sgs;             // Cp/Pr, Cp/Pr_sgs
  double C_s;
  double kappa2, kappa4, sigma;
  double gm1_half, mu_sut;          // (gamma - 1) / 2, mu_ref (1 + S_hat)
  int sigma_is_two_thirds;
  double cfl, dt_fixed;
  double p_inf;
  double jet_mach, theta_mom;
};

// Derived constants from the caller's parameters.
inline Consts make_consts(const jz_params& p) {
  Consts c;
  c.gamma = p.gamma;
  c.gm1 = p.gamma - 1.0;
  c.Cp = 1.0 / c.gm1;
  c.mu_ref = p.mach_ref / p.Re;
  c.S_hat = p.S1_K / p.T_ref_K;
  c.sut_num = 1.0 + c.S_hat;
  c.k_lam = c.Cp / p.Pr;
  c.k_sgs = c.Cp / p.Pr_sgs;
  c.C_s = p.C_s;
  c.kappa2 = p.kappa2;
  c.kappa4 = p.kappa4;
  c.gm1_half = 0.5 * c.gm1;
  c.mu_sut = c.mu_ref * c.sut_num;
  c.sigma = p.sigma;
  c.sigma_is_two_thirds = fabs(p.sigma - 2.0 / 3.0) < 1e-15 ? 1 : 0;
  c.cfl = p.cfl;
  c.dt_fixed = p.dt_fixed;
  c.p_inf = 1.0 / p.gamma;
  c.jet_mach = p.jet_mach;
  c.theta_mom = p.theta_mom;
  return c;
}

// Device scalars of a solver (one allocation).
struct Scalars {
  double t;          // time at the start of the current step
  double dt;         // current time step
  double rate_max;   // max over advanced nodes of (sum lambda)/V (as bits)
  double res_sum;    // sum of RHS_rho^2 at stage 1
  double tot[5];
  double min_rho, min_p;
  int nonfinite;
  int wait_timeout;   // set by a kernel whose bounded wait on an asynchronous copy ran out
};

// CFL rate of one node, (lambda_xi + lambda_eta + lambda_zeta) / V with
// lambda_d = |S^d . u| + a |S^d|, from its conserved variables: the stand-alone
// reduction (first FP32-flux step after jz_set_state, the adjoint's frozen step).
// The FP64 form's stage-1 nodal pass forms the same expressions from the same
// primitives.
__device__ __forceinline__ double node_rate(const GridDev& g, const Consts& c, long long p, double rho, double m1,
                                            double m2, double m3, double e) {
  const double ir = rcp64(rho);
  const double u = m1 * ir, v = m2 * ir, w = m3 * ir;
  const double pr = fma(-c.gm1_half, m1 * u + m2 * v + m3 * w, c.gm1 * e);   // (gamma-1)(e - rho|u|^2/2)
  const double a = sqrt64(c.gamma * pr * ir);
  double lsum = 0.0;
  if (!g.compact) {
    for (int dir = 0; dir < 3; ++dir) {
      const double U = g.S[3 * dir][p] * u + g.S[3 * dir + 1][p] * v + g.S[3 * dir + 2][p] * w;
      const double lam = fabs(U) + a * g.Smag[dir][p];
      lsum = dir == 0 ? lam : lsum + lam;
    }
    return lsum * g.invV[p];
  }
  // compact grid: the same rate from the FP32 metrics, widened
  const float* M = g.Mf + p * kMF;
  for (int dir = 0; dir < 3; ++dir) {
    const double sx = M[3 * dir], sy = M[3 * dir + 1], sz = M[3 * dir + 2];
    const double lam = fabs(sx * u + sy * v + sz * w) + a * sqrt64(sx * sx + sy * sy + sz * sz);
    lsum = dir == 0 ? lam : lsum + lam;
  }
  return lsum * (double)M[MF_IV];
}

// FP64 stage scratch arrays (each Np elements).
struct Work64 {
  double* u; double* v; double* w; double* T; double* p; double* mu;
  double* Lam[3];
  double* H[3][5];    // transformed inviscid flux, then inviscid - viscous
  double* nu[3];      // pressure sensor per direction
  double* G[3][5];    // twice the total face flux at n + 1/2: H_n + H_(n+1) - 2 d_(n+1/2)
};

// Pair form (JZ_PREC_FP64PAIR): double-float copies of the metrics (float2 hi/lo per padded
// node) and of the stage input Q (in FP64-sized arrays, two FP32 each).
struct DFMetrics {
  float2* S[9];
  float2* Smag[3];
  float2* invV;
  float2* Delta;
};
struct QDF {
  double* q[5];
};

struct State {
  double* q[5];
  // FP32-flux form only: the FP32 shadow of q, three float2 arrays of Np padded nodes
  // [(rho - 1, e - e_inf), (rho u, rho v), (rho w, p - p_inf)] (null in the FP64 form)
  float2* sh;
};

// Adjoint arrays (each Np elements unless noted).
struct Adj64 {
  double* lam[5];          // running adjoint of the stage state (real nodes; P0 as scratch)
  double* qnbar[5];        // adjoint of Q^n collected over the stages of a step
  double* acc[5];          // -(alpha dt / V) lam on advanced nodes, 0 elsewhere
  double* ca2[3];          // face coefficient Lambda_f eps2: the face adjoint of Q_{n+1} - Q_n
                           // is (acc_{n+1} - acc_n) ca2, that of the third difference
  double* ca4[3];          // -(acc_{n+1} - acc_n) ca4 with ca4 = Lambda_f eps4
  double* lfh[3];          // half the adjoint of the face spectral radius
  double* nb0[3];          // sensor adjoint sent to node n of face n+1/2
  double* nb1[3];          // ... and to node n+1
  double* G[4][3];         // adjoint of delta_dir f, f = u, v, w, T
  double* cpm[3];          // sensor adjoint coefficient of p_{n+1} and p_{n-1}
  double* c0[3];           // ... of p_n
  double* ubd[3];          // direct adjoint of u_i from the viscous energy flux
  double* mub;             // adjoint of the Sutherland viscosity
  double* rhob;            // direct adjoint of rho (eddy viscosity)
  double* abar;            // [32] dJ/dA accumulator
  double* J;               // [1] functional accumulator
};

// Inflow tables (jet): base profile u0[nk][nj] and forcing shapes
// Gf[m*4+f][nk][nj] = g(r) cos(m theta + phi_mf), at i = 0.
struct Inflow {
  double* u0;
  double* Gf;
  double amp[kNF];
  double psi[kNF];
  double omega[JZ_N_FREQ];       // 2 pi St_f U_j
};

// ---- kernels' host launchers -------------------------------------------
// metrics
cudaError_t pad_coordinates(const Dims& d, const double* xyz_real, const double* period,
                            GridDev& g, cudaStream_t st);
cudaError_t compute_metrics(const Dims& d, GridDev& g, double* scratch9[9], cudaStream_t st);
// ghost fill of nvar padded fields by the state's ghost map
cudaError_t ghost_fill(const Dims& d, double* const* f, int nvar, cudaStream_t st);
// FP32 copy of the metrics S (9) and V; dst_dev is a device array of 10 pointers
cudaError_t boundary_copies(const Dims& d, const GridDev& g, cudaStream_t st);
cudaError_t metrics_to_f32(const Dims& d, const GridDev& g, float* Mf, cudaStream_t st);
// copy between unpadded [nvar][N] and padded real region
cudaError_t pack_real(const Dims& d, double* const* padded, const double* flat, int nvar,
                      cudaStream_t st);
cudaError_t unpack_real(const Dims& d, double* const* padded, double* flat, int nvar,
                        cudaStream_t st);
// FP64 stage passes (one kernel each)
// rate_max != nullptr: also reduce the CFL rate of qin over the advanced nodes into
// *rate_max (max of (sum_dir lambda_dir) / V; the caller has left it 0)
cudaError_t nodal64(const Dims& d, const Consts& c, const GridDev& g, const Work64& w, const State& qin,
                    cudaStream_t st, double* rate_max = nullptr);
cudaError_t viscous64(const Dims& d, const Consts& c, const GridDev& g, const Work64& w, const State& qin,
                      cudaStream_t st);
cudaError_t faces64(const Dims& d, const Consts& c, const Work64& w, const State& qin, cudaStream_t st);
// stage update (rhs_flat == nullptr) or RHS output to rhs_flat [5][N]
cudaError_t update64(const Dims& d, const GridDev& g, const Work64& w, const State& qin, const State& qn,
                     const State& qout, const Scalars* sc, double alpha, int want_res, double* rhs_flat,
                     cudaStream_t st);
// FP32-flux stage (one fused kernel); Mf = the FP32 metric records (kMF floats per padded node);
// tm_in = the tensor map of qin's shadow (make_shadow_map).  The stage reads qin's shadow and
// writes qout and its shadow (or, with rhs_flat, the RHS only).
cudaError_t fused32(const Dims& d, const Consts& c, const float* Mf, const State& qin, const void* tm_in,
                    const State& qn, const State& qout, Scalars* sc, double alpha, int want_res, int want_rate,
                    double* rhs_flat, int kchunk, cudaStream_t st);
// FP32 shadow of q from its FP64 values: every padded node (full) or only the shell that the
// boundary conditions and the ghost fill rewrite after a stage (ghost layers and the planes
// i = 0, ni-1, j = 0, nj-1).
cudaError_t shadow_refresh(const Dims& d, const Consts& c, const State& q, int full, cudaStream_t st);
// TMA descriptor (CUtensorMap, 128 bytes, 64-byte aligned) of a shadow: 4-D (Pi, Pj, Pk, 3)
// of 8-byte elements; returns cudaErrorInvalidValue if the encoder is unavailable or refuses.
cudaError_t make_shadow_map(const Dims& d, float2* sh, void* tmap128);
cudaError_t fused32_slots(int* slots);
// self-check of the fused kernel's bounded mbarrier wait (jz_check_wait)
cudaError_t wait_check(int* dev_timed_out, long long* dev_cycles, cudaStream_t st);
int fused32_tile_x();
int fused32_tile_y();
// Pair form of the FP64 stage (jz_stagedf.cu): the four passes in double-float arithmetic,
// the stage combination in FP64.
cudaError_t metrics_to_df(const Dims& d, const GridDev& g, const DFMetrics& M, cudaStream_t st);
cudaError_t nodal_df(const Dims& d, const Consts& c, const DFMetrics& M, const Work64& w, const QDF& qdf,
                     const State& qin, cudaStream_t st, double* rate_max = nullptr);
cudaError_t viscous_df(const Dims& d, const Consts& c, const DFMetrics& M, const Work64& w, const QDF& qdf,
                       cudaStream_t st);
cudaError_t faces_update_df(const Dims& d, const Consts& c, const GridDev& g, const Work64& w, const QDF& qdf,
                            const State& qin, const State& qn, const State& qout, const Scalars* sc, double alpha,
                            int want_res, double* rhs_flat, cudaStream_t st);
// boundary conditions (jet), in this order after every stage
cudaError_t bc_farfield(const Dims& d, const Consts& c, const GridDev& g, const State& q, cudaStream_t st);
cudaError_t bc_inout(const Dims& d, const Consts& c, const Inflow& in, const State& q, const Scalars* sc,
                     double alpha, cudaStream_t st);
cudaError_t bc_axis(const Dims& d, const State& q, cudaStream_t st);
cudaError_t build_inflow(const Dims& d, const Consts& c, const GridDev& g, const jz_params& p,
                         Inflow& in, cudaStream_t st);
// reductions
cudaError_t cfl_rate(const Dims& d, const Consts& c, const GridDev& g, const State& q,
                     Scalars* sc, cudaStream_t st);
cudaError_t set_dt(const Consts& c, Scalars* sc, int advance_time, cudaStream_t st);
int stat_partial_count();
cudaError_t stats_with(const Dims& d, const Consts& c, const GridDev& g, const State& q, Scalars* sc,
                       double* part, cudaStream_t st);
cudaError_t check_volume(const Dims& d, const GridDev& g, int* bad, cudaStream_t st);
// self-check of rcp64 / cbrt64 (jz_mathcheck.cu)
cudaError_t math_check(double* dev_maxrel3, cudaStream_t st);
// self-check of the double-float operations of the pair form (jz_mathcheck.cu)
cudaError_t df_check(double* dev_maxrel9, cudaStream_t st);
// flow statistics of the axial velocity (jz_stats.cu)
cudaError_t flow_sample(const Dims& d, const State& q, double* mean, double* m2, long long n, cudaStream_t st);
cudaError_t flow_final(const Dims& d, const double* mean, const double* m2, long long n, double* out_mean,
                       double* out_rms, cudaStream_t st);

// adjoint (jz_adjoint.cu)
cudaError_t adj_update(const Dims& d, const GridDev& g, const Adj64& a, double adt, cudaStream_t st);
// mdf, qdf non-null: a pair-form solver, whose forward intermediates in w are double-float pairs;
// its transposed face, viscous and nodal passes run in pair arithmetic (adj_faces_df,
// adj_visc_df, adj_nodal_df, jz_adjointdf.cu)
cudaError_t adj_stage(const Dims& d, const Consts& c, const GridDev& g, const Work64& w, const State& q,
                      const Adj64& a, const DFMetrics* mdf, const QDF* qdf, cudaStream_t st);
cudaError_t adj_visc_df(const Dims& d, const Consts& c, const DFMetrics& M, const Work64& w, const QDF& qdf,
                        const Adj64& a, cudaStream_t st);
cudaError_t adj_faces_df(const Dims& d, const Consts& c, const Work64& w, const QDF& qdf, const Adj64& a,
                         cudaStream_t st);
cudaError_t adj_nodal_df(const Dims& d, const Consts& c, const DFMetrics& M, const QDF& qdf, const Adj64& a,
                         cudaStream_t st);
// pair-form solver: acc stored as double-float pairs (read by the pair transposed passes only)
cudaError_t adj_update_df(const Dims& d, const GridDev& g, const Adj64& a, double adt, cudaStream_t st);
cudaError_t adj_add_qn(const Dims& d, const Adj64& a, cudaStream_t st);
cudaError_t adj_bcs(const Dims& d, const Consts& c, const GridDev& g, const Inflow& in, const State& q,
                    const Adj64& a, double ts, cudaStream_t st);
cudaError_t observer(const Dims& d, const Consts& c, const State& q, const double* w, int j0, double beta,
                     double dt, const Adj64& a, int want_grad, cudaStream_t st);
cudaError_t set_time(Scalars* sc, double t, double dt, cudaStream_t st);

// ---- shared with the C ABI layer ------------------------------------------
// Record an error message for jz_last_error(); returns code.
int set_error(int code, const char* msg);
// Dimensions and device arrays of a grid whose metrics are computed.
bool grid_view(const jz_grid* g, Dims* d, GridDev* dev);

// ---- helpers ------------------------------------------------------------
inline unsigned blocks_for(long long n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

// Flat thread index over a box [i0, i0+ei) x [j0, j0+ej) x [k0, k0+ek) of
// real coordinates; returns false past the end.
struct Box {
  int i0, j0, k0, ei, ej, ek;
  long long count() const { return (long long)ei * ej * ek; }
};

__device__ inline bool box_coord(const Box& b, long long t, int& i, int& j, int& k) {
  if (t >= (long long)b.ei * b.ej * b.ek) return false;
  i = (int)(t % b.ei);
  long long r = t / b.ei;
  j = (int)(r % b.ej);
  k = (int)(r / b.ej);
  i += b.i0; j += b.j0; k += b.k0;
  return true;
}

// Real node whose state a padded node carries (the ghost map).
__host__ __device__ inline void ghost_source(const Dims& d, int i, int j, int k, int& si, int& sj,
                                             int& sk) {
  if (d.topo == JZ_TOPO_PERIODIC) {
    si = ((i % d.ni) + d.ni) % d.ni;
    sj = ((j % d.nj) + d.nj) % d.nj;
    sk = ((k % d.nk) + d.nk) % d.nk;
    return;
  }
  si = i < 0 ? 0 : (i >= d.ni ? d.ni - 1 : i);
  int kk = k;
  if (j < 0) { sj = -j; kk = k + d.nk / 2; }
  else if (j >= d.nj) { sj = d.nj - 1; }
  else { sj = j; }
  sk = ((kk % d.nk) + d.nk) % d.nk;
}

}  // namespace jz
