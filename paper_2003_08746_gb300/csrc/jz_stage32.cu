// FP32-flux form of one Runge-Kutta stage: fluxes, dissipation and SGS terms
// in FP32; the state Q, the stage combination Q^n - alpha dt RHS and the
// totals in FP64.  One fused kernel per stage, one HBM sweep:
//
//   read Q^(l-1) (FP64, halo 2), Q^n (FP64, own node), metrics (FP32, halo 1),
//   write Q^(l) (FP64).
//
// Each CTA owns a TX x TY tile of (i, j) columns and marches in k.  Shared
// memory holds a ring of three planes of FP32 primitives (tile + 2-node
// halo) and a ring of two planes of nodal fluxes, spectral radii and
// sensors (tile + 1-node halo).  Per plane:
//   (a) the FP64 state of plane k+2 (prefetched into registers one plane
//       earlier) is converted to FP32 and reduced to primitives,
//   (b) every node of plane k+1 within one node of the tile gets its
//       gradients, viscous and inviscid transformed fluxes H^dir, spectral
//       radii Lambda^dir and pressure sensors nu^dir,
//   (c) the tile of plane k gets its dissipation faces, RHS and update.
//
// On a GB300 the FP64 pipe (DADD/DFMA, and also the F2F conversions between
// FP64 and FP32) issues ~2 instructions per SM per clock against 128 for
// FP32, so FP64 -> FP32 conversions are done with integer bit operations
// (truncation), and FP32 -> FP64 exactly, also with integer operations.
// Only the offsets rho - 1, e - e_inf (which keep the FP32 values small in
// the ambient flow) and the final Q^n - dQ are FP64 additions.
#include "jz_internal.cuh"

namespace jz {
namespace {

#ifndef JZ_FUSED_TX
#define JZ_FUSED_TX 30
#endif
#ifndef JZ_FUSED_TY
#define JZ_FUSED_TY 8
#endif
constexpr int TX = JZ_FUSED_TX, TY = JZ_FUSED_TY;
constexpr int H1X = TX + 2, H1Y = TY + 2, NP1 = H1X * H1Y;   // 32 x 10
constexpr int H2X = TX + 4, H2Y = TY + 4, NP2 = H2X * H2Y;   // 34 x 12
constexpr int NT = NP1;                                      // threads per CTA
constexpr int NOUT = TX * TY;
constexpr int NLOAD = (NP2 + NT - 1) / NT;                   // halo-2 points per thread

// primitive ring: rho' = rho - 1, m1, m2, m3, e' = e - e_inf, u, v, w, T, p' = p - p_inf
constexpr int F_R = 0, F_E = 4, F_U = 5, F_V = 6, F_W = 7, F_T = 8, F_P = 9, NPF = 10;
// flux ring: H^xi(5), H^eta(5), H^zeta(5), Lambda(3), nu(3), 1/V
constexpr int G_HX = 0, G_HY = 5, G_HZ = 10, G_L = 15, G_N = 18, G_IV = 21, NGF = 22;

struct Smem {
  float prim[3][NPF][NP2];
  float flux[2][NGF][NP1];
};

struct ConstsF {
  float gamma, gm1, mu_ref, S_hat, sut_num, k_lam, k_sgs, C_s, kappa2, kappa4;
  float p_inf, ep_inf;     // p_inf, e_inf + p_inf
  double e_inf;            // p_inf / (gamma - 1), subtracted in FP64
};

// FP64 -> FP32 by bit manipulation (truncation toward zero; magnitudes below
// 2^-126 flush to signed zero).  Valid for finite |x| < 2^128.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e8 = (int)((hi >> 20) & 0x7FFu) - 896;
  const unsigned m = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
  const unsigned s = hi & 0x80000000u;
  return __uint_as_float(e8 > 0 ? (s | ((unsigned)e8 << 23) | m) : s);
}

// FP32 -> FP64, exact (subnormals flush to zero; Inf/NaN kept).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u, e8 = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (e8 == 0) return __hiloint2double((int)s, 0);
  const unsigned e11 = e8 == 0xFFu ? 0x7FFu : e8 + 896u;
  return __hiloint2double((int)(s | (e11 << 20) | (m >> 3)), (int)(m << 29));
}

// Single MUFU approximations (relative error ~2^-22), far inside the FP32-flux
// form's error budget.
__device__ __forceinline__ float f_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float f_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float f_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float f_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float cbrt_pos(float x) {   // x >= 0; 0 -> 0
  return x > 0.f ? f_ex2(f_lg2(x) * (1.f / 3.f)) : 0.f;
}

__device__ __forceinline__ int ring3(int k) { return (k + 6) % 3; }   // k >= -6

__device__ __forceinline__ bool in_padded(const Dims& d, int i, int j) {
  return i >= -kG && i <= d.ni + 1 && j >= -kG && j <= d.nj + 1;
}

// Turkel-Vatsa face flux between nodes a and b = a + s (d = Lambda_f [eps2 dQ - eps4 d3Q]).
__device__ __forceinline__ void face_flux(const ConstsF& c, float La, float Lb, float na, float nb,
                                          const float qm[5], const float q0[5], const float q1[5],
                                          const float q2[5], float out[5]) {
  const float eps2 = c.kappa2 * fmaxf(na, nb);
  const float eps4 = fmaxf(0.f, c.kappa4 - eps2);
  const float Lf = 0.5f * (La + Lb);
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const float d1 = q1[m] - q0[m];
    const float d3 = (q2[m] - qm[m]) + 3.f * (q0[m] - q1[m]);
    out[m] = Lf * (eps2 * d1 - eps4 * d3);
  }
}

struct Args {
  Dims d;
  ConstsF c;
  const float* S[10];        // S^xi, S^eta, S^zeta (9), V, FP32
  const double* qin[5];
  const double* qn[5];
  double* qout[5];
  double* rhs;               // non-null: write RHS [5][N] instead of updating
  Scalars* sc;
  double alpha;
  int kchunk;
  int want_res;
  int want_rate;
};

// Padded index at k = 0 of this thread's halo-2 load points (-1: outside the padded box).
__device__ __forceinline__ void load_bases(const Args& A, int i0, int j0, long long base[NLOAD]) {
#pragma unroll
  for (int r = 0; r < NLOAD; ++r) {
    const int t = threadIdx.x + r * NT;
    const int i = i0 - 2 + t % H2X, j = j0 - 2 + t / H2X;
    base[r] = (t < NP2 && in_padded(A.d, i, j)) ? pidx(A.d, i, j, 0) : -1;
  }
}

// Load the FP64 state of plane k at this thread's halo-2 points into registers.
__device__ __forceinline__ void prefetch(const Args& A, const long long base[NLOAD], int k, double reg[NLOAD][5]) {
  const long long koff = (long long)k * A.d.sk;
#pragma unroll
  for (int r = 0; r < NLOAD; ++r) {
    if (base[r] >= 0) {
      const long long p = base[r] + koff;
#pragma unroll
      for (int m = 0; m < 5; ++m) reg[r][m] = __ldg(A.qin[m] + p);
    } else {
      reg[r][0] = 1.0; reg[r][1] = 0.0; reg[r][2] = 0.0; reg[r][3] = 0.0; reg[r][4] = A.c.e_inf;
    }
  }
}

// Convert prefetched FP64 state to FP32 primitives in a ring slot.
__device__ __forceinline__ void store_prims(const Args& A, Smem& sm, int slot, const double reg[NLOAD][5]) {
  const ConstsF& c = A.c;
#pragma unroll
  for (int r = 0; r < NLOAD; ++r) {
    const int t = threadIdx.x + r * NT;
    if (t < NP2) {
      const float rp = f64_to_f32(reg[r][0] - 1.0);
      const float m1 = f64_to_f32(reg[r][1]), m2 = f64_to_f32(reg[r][2]), m3 = f64_to_f32(reg[r][3]);
      const float ep = f64_to_f32(reg[r][4] - c.e_inf);
      const float rho = rp + 1.f;
      const float ir = f_rcp(rho);
      const float u = m1 * ir, v = m2 * ir, w = m3 * ir;
      const float pp = c.gm1 * (ep - 0.5f * (m1 * u + m2 * v + m3 * w));
      const float T = c.gamma * (pp + c.p_inf) * ir;
      float* P = &sm.prim[slot][0][0];
      P[F_R * NP2 + t] = rp;
      P[1 * NP2 + t] = m1;
      P[2 * NP2 + t] = m2;
      P[3 * NP2 + t] = m3;
      P[F_E * NP2 + t] = ep;
      P[F_U * NP2 + t] = u;
      P[F_V * NP2 + t] = v;
      P[F_W * NP2 + t] = w;
      P[F_T * NP2 + t] = T;
      P[F_P * NP2 + t] = pp;
    }
  }
}

// Metrics S (9) and V of this thread's halo-1 node of plane q (nb < 0: outside).
__device__ __forceinline__ void load_metrics(const Args& A, long long nb, int q, float met[10]) {
  if (nb < 0) {
#pragma unroll
    for (int f = 0; f < 10; ++f) met[f] = 0.f;
    return;
  }
  const long long p = nb + (long long)q * A.d.sk;
#pragma unroll
  for (int f = 0; f < 10; ++f) met[f] = __ldg(A.S[f] + p);
}

// Nodal fluxes, spectral radii and sensors of one node of plane q (slots
// s_m, s_0, s_p of planes q-1, q, q+1) at halo-1 index t.
__device__ void nodal(const Args& A, Smem& sm, long long nb, const float met[10], int s_m, int s_0, int s_p, int g) {
  const ConstsF& c = A.c;
  const int t = threadIdx.x;
  const int x1 = t % H1X, y1 = t / H1X;
  const int c2 = (y1 + 1) * H2X + (x1 + 1);
  float* Fo = &sm.flux[g][0][0];
  if (nb < 0) {
#pragma unroll 1
    for (int f = 0; f < NGF; ++f) Fo[f * NP1 + t] = 0.f;
    return;
  }
  float S[3][3];
#pragma unroll
  for (int dir = 0; dir < 3; ++dir)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) S[dir][cc] = met[3 * dir + cc];
  const float V = met[9];
  const float iV = V > 0.f ? f_rcp(V) : 0.f;
  const float* P0 = &sm.prim[s_0][0][0];
  const float* Pm = &sm.prim[s_m][0][0];
  const float* Pp = &sm.prim[s_p][0][0];
  // gradients of u, v, w, T: L[n][jj] = (1/V) sum_dir S^dir_jj delta_dir f_n
  float L[4][3];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int f = F_U + n;
    const float dx = 0.5f * (P0[f * NP2 + c2 + 1] - P0[f * NP2 + c2 - 1]);
    const float dy = 0.5f * (P0[f * NP2 + c2 + H2X] - P0[f * NP2 + c2 - H2X]);
    const float dz = 0.5f * (Pp[f * NP2 + c2] - Pm[f * NP2 + c2]);
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) L[n][jj] = iV * (S[0][jj] * dx + S[1][jj] * dy + S[2][jj] * dz);
  }
  const float rho = P0[F_R * NP2 + c2] + 1.f;
  const float m1 = P0[1 * NP2 + c2], m2 = P0[2 * NP2 + c2], m3 = P0[3 * NP2 + c2];
  const float u = P0[F_U * NP2 + c2], v = P0[F_V * NP2 + c2], w = P0[F_W * NP2 + c2];
  const float T = P0[F_T * NP2 + c2], pp = P0[F_P * NP2 + c2];
  const float ep = P0[F_E * NP2 + c2];
  const float a = f_sqrt(T);
  const float mu = c.mu_ref * (T * a) * c.sut_num * f_rcp(T + c.S_hat);
  float Sij[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) Sij[x][y] = 0.5f * (L[x][y] + L[y][x]);
  const float div = Sij[0][0] + Sij[1][1] + Sij[2][2];
  float SS = 0.f;
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) SS += Sij[x][y] * Sij[x][y];
  const float Smod = f_sqrt(2.f * SS);
  const float csd = c.C_s * cbrt_pos(V);
  const float mu_sgs = rho * (csd * csd) * Smod;
  const float mu_eff = mu + mu_sgs;
  const float k_eff = mu * c.k_lam + mu_sgs * c.k_sgs;
  const float d3 = div * (1.f / 3.f);
  float tau[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) tau[x][y] = 2.f * mu_eff * (Sij[x][y] - (x == y ? d3 : 0.f));
  float F[3][4];
#pragma unroll
  for (int jj = 0; jj < 3; ++jj) {
    F[jj][0] = tau[0][jj];
    F[jj][1] = tau[1][jj];
    F[jj][2] = tau[2][jj];
    F[jj][3] = u * tau[0][jj] + v * tau[1][jj] + w * tau[2][jj] + k_eff * L[3][jj];
  }
  const float h0 = ep + pp + c.ep_inf;   // e + p
  float lam[3];
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    const float U = S[dir][0] * u + S[dir][1] * v + S[dir][2] * w;
    const float smag = f_sqrt(S[dir][0] * S[dir][0] + S[dir][1] * S[dir][1] + S[dir][2] * S[dir][2]);
    lam[dir] = fabsf(U) + a * smag;
    const int gh = G_HX + 5 * dir;
    Fo[(gh + 0) * NP1 + t] = rho * U;
    const float fv0 = S[dir][0] * F[0][0] + S[dir][1] * F[1][0] + S[dir][2] * F[2][0];
    const float fv1 = S[dir][0] * F[0][1] + S[dir][1] * F[1][1] + S[dir][2] * F[2][1];
    const float fv2 = S[dir][0] * F[0][2] + S[dir][1] * F[1][2] + S[dir][2] * F[2][2];
    const float fv3 = S[dir][0] * F[0][3] + S[dir][1] * F[1][3] + S[dir][2] * F[2][3];
    Fo[(gh + 1) * NP1 + t] = m1 * U + pp * S[dir][0] - fv0;
    Fo[(gh + 2) * NP1 + t] = m2 * U + pp * S[dir][1] - fv1;
    Fo[(gh + 3) * NP1 + t] = m3 * U + pp * S[dir][2] - fv2;
    Fo[(gh + 4) * NP1 + t] = h0 * U - fv3;
  }
  const float t0 = cbrt_pos(lam[0]), t1 = cbrt_pos(lam[1]), t2 = cbrt_pos(lam[2]);
  Fo[(G_L + 0) * NP1 + t] = lam[0] + t0 * (t1 * t1 + t2 * t2);
  Fo[(G_L + 1) * NP1 + t] = lam[1] + t1 * (t0 * t0 + t2 * t2);
  Fo[(G_L + 2) * NP1 + t] = lam[2] + t2 * (t0 * t0 + t1 * t1);
  // pressure sensors (p' = p - p_inf; denominators add 4 p_inf back)
  const float* pr0 = P0 + F_P * NP2;
  const float pxm = pr0[c2 - 1], pxp = pr0[c2 + 1], pym = pr0[c2 - H2X], pyp = pr0[c2 + H2X];
  const float pzm = Pm[F_P * NP2 + c2], pzp = Pp[F_P * NP2 + c2];
  const float p4 = 4.f * c.p_inf;
  Fo[(G_N + 0) * NP1 + t] = fabsf(pxp - 2.f * pp + pxm) * f_rcp(pxp + 2.f * pp + pxm + p4);
  Fo[(G_N + 1) * NP1 + t] = fabsf(pyp - 2.f * pp + pym) * f_rcp(pyp + 2.f * pp + pym + p4);
  Fo[(G_N + 2) * NP1 + t] = fabsf(pzp - 2.f * pp + pzm) * f_rcp(pzp + 2.f * pp + pzm + p4);
  Fo[G_IV * NP1 + t] = iV;
}

__device__ __forceinline__ void load_q(const float* P, int c2, float q[5]) {
#pragma unroll
  for (int m = 0; m < 5; ++m) q[m] = P[m * NP2 + c2];
}

constexpr int kMinBlocks = NT <= 320 ? 2 : 1;

__global__ void __launch_bounds__(NT, kMinBlocks) k_fused32(Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  const Dims& d = A.d;
  const ConstsF& c = A.c;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * A.kchunk;
  const int k1 = min(k0 + A.kchunk, d.nk);          // output planes [k0, k1)
  const int t = threadIdx.x;
  const bool outth = t < NOUT;
  const int ox = t % TX, oy = t / TX;
  const int oi = i0 + ox, oj = j0 + oy;
  const bool outv = outth && oi < d.ni && oj < d.nj;
  const bool adv = outv && (d.topo != JZ_TOPO_JET || (oi >= 1 && oi <= d.ni - 2 && oj >= 1 && oj <= d.nj - 2));
  const int c1 = (oy + 1) * H1X + (ox + 1);
  const int c2 = (oy + 2) * H2X + (ox + 2);

  long long lb[NLOAD];
  load_bases(A, i0, j0, lb);
  long long nb;                                    // halo-1 node of this thread (nodal work)
  {
    const int i = i0 - 1 + t % H1X, j = j0 - 1 + t / H1X;
    nb = in_padded(d, i, j) ? pidx(d, i, j, 0) : -1;
  }
  const long long ob = outv ? pidx(d, oi, oj, 0) : 0;   // output node
  double reg[NLOAD][5];
  // prime: planes k0-2, k0-1 into the ring, plane k0 into registers
  prefetch(A, lb, k0 - 2, reg);
  store_prims(A, sm, ring3(k0 - 2), reg);
  prefetch(A, lb, k0 - 1, reg);
  store_prims(A, sm, ring3(k0 - 1), reg);
  prefetch(A, lb, k0, reg);

  float Hz_prev[5] = {0, 0, 0, 0, 0};   // H^zeta(p-1)
  float Dz_prev[5] = {0, 0, 0, 0, 0};   // d^zeta(p-1/2)
  float Qz_prev[5] = {0, 0, 0, 0, 0};   // Q(p-1), FP32
  float Lz = 0.f, Nz = 0.f;             // Lambda^zeta(p), nu^zeta(p)
  const float adt = f64_to_f32(A.alpha * A.sc->dt);
  float res = 0.f, rate = 0.f;

  for (int p = k0 - 2; p < k1; ++p) {
    // (a) metrics of plane p+1 (used in (b)); plane p+2 -> ring; prefetch plane p+3
    float met[10];
    load_metrics(A, nb, p + 1, met);
    store_prims(A, sm, ring3(p + 2), reg);
    if (p + 3 <= k1 + 1) prefetch(A, lb, p + 3, reg);
    __syncthreads();
    // (b) nodal quantities of plane p+1
    nodal(A, sm, nb, met, ring3(p), ring3(p + 1), ring3(p + 2), (p + 1) & 1);
    __syncthreads();
    // (c) zeta face p+1/2 and the output plane p
    if (outth) {
      const float* Fp1 = &sm.flux[(p + 1) & 1][0][0];
      const float* P0 = &sm.prim[ring3(p)][0][0];
      const float* P1 = &sm.prim[ring3(p + 1)][0][0];
      const float* P2 = &sm.prim[ring3(p + 2)][0][0];
      const float Lz1 = Fp1[(G_L + 2) * NP1 + c1], Nz1 = Fp1[(G_N + 2) * NP1 + c1];
      float q0[5], q1[5], q2[5], Dz[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      load_q(P0, c2, q0);
      load_q(P1, c2, q1);
      load_q(P2, c2, q2);
      if (p >= k0 - 1) face_flux(c, Lz, Lz1, Nz, Nz1, Qz_prev, q0, q1, q2, Dz);
      if (p >= k0 && outv) {
        const float* F0 = &sm.flux[p & 1][0][0];
        float R[5];
        // xi faces i -/+ 1/2 and eta faces j -/+ 1/2
        float a0[5], a1[5], a2[5], a3[5], Dxm[5], Dxp[5], Dym[5], Dyp[5];
        load_q(P0, c2 - 2, a0); load_q(P0, c2 - 1, a1); load_q(P0, c2 + 1, a2); load_q(P0, c2 + 2, a3);
        face_flux(c, F0[G_L * NP1 + c1 - 1], F0[G_L * NP1 + c1], F0[G_N * NP1 + c1 - 1], F0[G_N * NP1 + c1],
                  a0, a1, q0, a2, Dxm);
        face_flux(c, F0[G_L * NP1 + c1], F0[G_L * NP1 + c1 + 1], F0[G_N * NP1 + c1], F0[G_N * NP1 + c1 + 1],
                  a1, q0, a2, a3, Dxp);
        load_q(P0, c2 - 2 * H2X, a0); load_q(P0, c2 - H2X, a1); load_q(P0, c2 + H2X, a2);
        load_q(P0, c2 + 2 * H2X, a3);
        face_flux(c, F0[(G_L + 1) * NP1 + c1 - H1X], F0[(G_L + 1) * NP1 + c1], F0[(G_N + 1) * NP1 + c1 - H1X],
                  F0[(G_N + 1) * NP1 + c1], a0, a1, q0, a2, Dym);
        face_flux(c, F0[(G_L + 1) * NP1 + c1], F0[(G_L + 1) * NP1 + c1 + H1X], F0[(G_N + 1) * NP1 + c1],
                  F0[(G_N + 1) * NP1 + c1 + H1X], a1, q0, a2, a3, Dyp);
        const float iV = F0[G_IV * NP1 + c1];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          float acc = 0.5f * (F0[(G_HX + m) * NP1 + c1 + 1] - F0[(G_HX + m) * NP1 + c1 - 1]) - (Dxp[m] - Dxm[m]);
          acc += 0.5f * (F0[(G_HY + m) * NP1 + c1 + H1X] - F0[(G_HY + m) * NP1 + c1 - H1X]) - (Dyp[m] - Dym[m]);
          acc += 0.5f * (Fp1[(G_HZ + m) * NP1 + c1] - Hz_prev[m]) - (Dz[m] - Dz_prev[m]);
          R[m] = acc * iV;
        }
        const long long pp = ob + (long long)p * d.sk;
        if (A.rhs) {
          const long long N = (long long)d.ni * d.nj * d.nk;
          const long long ridx = ((long long)p * d.nj + oj) * d.ni + oi;
#pragma unroll
          for (int m = 0; m < 5; ++m) A.rhs[m * N + ridx] = adv ? f32_to_f64(R[m]) : 0.0;
        } else if (adv) {
          double qnew[5];
#pragma unroll
          for (int m = 0; m < 5; ++m) {
            qnew[m] = __ldg(A.qn[m] + pp) - f32_to_f64(adt * R[m]);
            A.qout[m][pp] = qnew[m];
          }
          if (A.want_rate) {
            const float rho = f64_to_f32(qnew[0]);
            const float ir = f_rcp(rho);
            const float m1 = f64_to_f32(qnew[1]), m2 = f64_to_f32(qnew[2]), m3 = f64_to_f32(qnew[3]);
            const float u = m1 * ir, v = m2 * ir, w = m3 * ir;
            const float pr = c.gm1 * (f64_to_f32(qnew[4] - c.e_inf) - 0.5f * (m1 * u + m2 * v + m3 * w)) + c.p_inf;
            const float a = f_sqrt(c.gamma * pr * ir);
            float ls = 0.f;
#pragma unroll
            for (int dir = 0; dir < 3; ++dir) {
              const float sx = __ldg(A.S[3 * dir] + pp), sy = __ldg(A.S[3 * dir + 1] + pp),
                          sz = __ldg(A.S[3 * dir + 2] + pp);
              ls += fabsf(sx * u + sy * v + sz * w) + a * f_sqrt(sx * sx + sy * sy + sz * sz);
            }
            rate = fmaxf(rate, ls * iV);
          }
        } else {
#pragma unroll
          for (int m = 0; m < 5; ++m) A.qout[m][pp] = A.qin[m][pp];
        }
        if (adv) res += R[0] * R[0];
      }
      // rotate the zeta registers
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        Hz_prev[m] = sm.flux[p & 1][G_HZ + m][c1];
        Dz_prev[m] = Dz[m];
        Qz_prev[m] = q0[m];
      }
      Lz = Lz1;
      Nz = Nz1;
    }
    __syncthreads();
  }
  if (A.want_res || A.want_rate) {
    __shared__ float red[2][NT / 32];
    float r1 = res, r2 = rate;
    for (int o = 16; o > 0; o >>= 1) {
      r1 += __shfl_xor_sync(0xffffffffu, r1, o);
      r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    }
    if ((t & 31) == 0) { red[0][t >> 5] = r1; red[1][t >> 5] = r2; }
    __syncthreads();
    if (t == 0) {
      float s1 = 0.f, s2 = 0.f;
      for (int w = 0; w < NT / 32; ++w) { s1 += red[0][w]; s2 = fmaxf(s2, red[1][w]); }
      if (A.want_res) atomicAdd(&A.sc->res_sum, (double)s1);
      if (A.want_rate && s2 > 0.f)
        atomicMax(reinterpret_cast<unsigned long long*>(&A.sc->rate_max),
                  (unsigned long long)__double_as_longlong((double)s2));
    }
  }
}

}  // namespace

cudaError_t fused32(const Dims& d, const Consts& c, float* const* Sf, const State& qin, const State& qn,
                    const State& qout, Scalars* sc, double alpha, int want_res, int want_rate, double* rhs_flat,
                    int kchunk, cudaStream_t st) {
  static bool attr[64] = {false};     // the attribute is per device
  const int smem = (int)sizeof(Smem);
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return e0;
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_fused32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  Args A;
  A.d = d;
  A.c.gamma = (float)c.gamma; A.c.gm1 = (float)c.gm1; A.c.mu_ref = (float)c.mu_ref; A.c.S_hat = (float)c.S_hat;
  A.c.sut_num = (float)c.sut_num; A.c.k_lam = (float)c.k_lam; A.c.k_sgs = (float)c.k_sgs; A.c.C_s = (float)c.C_s;
  A.c.kappa2 = (float)c.kappa2; A.c.kappa4 = (float)c.kappa4; A.c.p_inf = (float)c.p_inf;
  A.c.e_inf = c.p_inf / c.gm1;
  A.c.ep_inf = (float)(A.c.e_inf + c.p_inf);
  for (int i = 0; i < 10; ++i) A.S[i] = Sf[i];
  for (int m = 0; m < 5; ++m) {
    A.qin[m] = qin.q[m];
    A.qn[m] = qn.q[m];
    A.qout[m] = qout.q[m];
  }
  A.rhs = rhs_flat;
  A.sc = sc;
  A.alpha = alpha;
  A.kchunk = kchunk > 0 ? kchunk : d.nk;
  A.want_res = want_res;
  A.want_rate = want_rate;
  dim3 grid((d.ni + TX - 1) / TX, (d.nj + TY - 1) / TY, (d.nk + A.kchunk - 1) / A.kchunk);
  k_fused32<<<grid, NT, smem, st>>>(A);
  return cudaGetLastError();
}

int fused32_tile_x() { return TX; }
int fused32_tile_y() { return TY; }

}  // namespace jz
