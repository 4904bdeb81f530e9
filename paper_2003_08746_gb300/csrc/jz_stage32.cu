// FP32-flux form of one Runge-Kutta stage: fluxes, dissipation and SGS terms
// in FP32; the state Q, the stage combination Q^n - alpha dt RHS and the
// totals in FP64.  One fused kernel per stage, one HBM sweep:
//
//   read the FP32 shadow of Q^(l-1) (halo 2, by TMA), Q^n (FP64, own node),
//   metrics (FP32, halo 1); write Q^(l) (FP64) and its FP32 shadow.
//
// The shadow of a state is what the stage's FP32 arithmetic reads of it, kept
// beside the FP64 state in three float2 arrays per padded node:
// (rho - 1, e - e_inf), (rho u, rho v), (rho w, p - p_inf).  The offsets keep
// the FP32 values small in the ambient flow.  The stage that writes Q^(l)
// writes its shadow; after the boundary conditions and the ghost fill a shell
// kernel refreshes the shadow of the nodes they rewrote.
//
// Each CTA owns a TX x TY tile of (i, j) columns and marches in k.  Shared
// memory holds a ring of four planes of the shadow (tile + 2-node halo; each
// plane is one 4-D TMA box of 34 x 12 x 1 x 3 float2 landing on an mbarrier),
// a ring of two planes of in-plane nodal fluxes, spectral radii and sensors
// (tile + 1-node halo), the same for the zeta direction (tile only), and the
// xi/eta dissipation faces of one plane.  Per plane:
//   (a) wait for the shadow of plane k+2 (requested one plane earlier) and
//       form 1/rho on its points; one thread then requests plane k+3,
//   (b) every node of plane k+1 within one node of the tile gets its
//       gradients, viscous and inviscid transformed fluxes H^dir, spectral
//       radii Lambda^dir and pressure sensors nu^dir; the same threads then
//       compute each xi and eta dissipation face of plane k once,
//   (c) the tile of plane k gets its zeta face, RHS and update.
//
// On a GB300 the FP64 pipe (DADD/DFMA, and also the F2F conversions between
// FP64 and FP32) issues ~2 instructions per SM per clock against 128 for
// FP32, so FP64 -> FP32 conversions are done with integer bit operations
// (truncation), and FP32 -> FP64 exactly, also with integer operations.
// Only the offsets rho - 1, e - e_inf and the final Q^n - dQ are FP64
// additions.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

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
constexpr int NOT = 32 * TY;                                 // output threads: one warp per row
static_assert(TX <= 32 && NOT <= NT, "one warp per output row");
constexpr int NIR = (NP2 + NT - 1) / NT;                     // halo-2 points per thread (1/rho pass)

// shadow ring: per halo-2 point three float2 pairs, as in global memory
// (rho' = rho - 1, e' = e - e_inf), (m1, m2), (m3, p' = p - p_inf), and 1/rho beside them
// (u = m/rho and T = gamma p/rho are formed where they are used)
constexpr int NSH = 3;
constexpr int NRING = 4;           // planes k-1 .. k+2: the next plane's request needs no barrier
constexpr int BOX_BYTES = NSH * NP2 * 8;                       // one TMA box (34 x 12 x 1 x 3 float2)
constexpr int SLOT = ((BOX_BYTES + 127) / 128) * 128 / 8;      // float2 per ring slot, 128-byte aligned
// in-plane flux ring (tile + 1 halo): H^xi(5), H^eta(5), Lambda^xi, Lambda^eta, nu^xi, nu^eta
constexpr int X_HX = 0, X_HY = 5, X_LX = 10, X_LY = 11, X_NX = 12, X_NY = 13, NXF = 14;
// zeta ring (tile): H^zeta(5), Lambda^zeta, nu^zeta, 1/V
constexpr int Z_HZ = 0, Z_L = 5, Z_N = 6, Z_IV = 7, NZF = 8;
// xi faces: TY rows of TX+1; eta faces: TY+1 rows of TX
constexpr int NFX = TY * (TX + 1), NFY = (TY + 1) * TX;

struct Smem {
  float2 sh[NRING][SLOT];          // TMA destinations (first member: 128-byte aligned)
  float ir[NRING][NP2];
  float fxy[2][NXF][NP1];
  float fz[2][NZF][NOUT];
  float dx[5][NFX];
  float dy[5][NFY];
  unsigned long long bar[NRING];   // one mbarrier per ring slot
  int fail;                        // a bounded wait ran out in this CTA
};

struct ConstsF {
  float gamma, gm1, mu_ref, S_hat, sut_num, k_lam, k_sgs, C_s, kappa2, kappa4;
  float p_inf, ep_inf;     // p_inf, e_inf + p_inf
  double e_inf;            // p_inf / (gamma - 1), subtracted in FP64
};

// FP64 -> FP32 by bit manipulation (truncation toward zero; magnitudes below
// 2^-126 flush to signed zero).  Valid for finite |x| < 2^128.  Re-biasing the
// exponent on the high word (e - 896 fits in 8 bits) lets one funnel shift pick
// the FP32 exponent and the top 23 mantissa bits at once.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned f = __funnelshift_l(lo, hi - (896u << 20), 3);
  const unsigned r = (f & 0x7FFFFFFFu) | (hi & 0x80000000u);
  return __uint_as_float((hi << 1) >= (897u << 21) ? r : (hi & 0x80000000u));
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
// Ask L2 to fetch the sector holding p (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ float cbrt_pos(float x) {   // x >= 0; 0 -> 0
  return x > 0.f ? f_ex2(f_lg2(x) * (1.f / 3.f)) : 0.f;
}

__device__ __forceinline__ int ring(int k) { return (k + 8) & (NRING - 1); }   // k >= -8

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
  // Lf (eps2 d1 - eps4 d3) with d3 = (q2 - qm) - 3 d1, as (Lf eps2 + 3 Lf eps4) d1 - Lf eps4 (q2 - qm)
  const float b = Lf * eps4;
  const float a3 = fmaf(3.f, b, Lf * eps2);
#pragma unroll
  for (int m = 0; m < 5; ++m) out[m] = fmaf(a3, q1[m] - q0[m], -b * (q2[m] - qm[m]));
}

struct Args {
  CUtensorMap tm;            // shadow of Q^(l-1): 4-D (Pi, Pj, Pk, 3) of float2, box 34 x 12 x 1 x 3
  Dims d;
  ConstsF c;
  const float* M;            // FP32 metric records, kMF floats per padded node
  const double* qin[5];      // FP64 Q^(l-1): copied on the nodes the stage does not advance
  const double* qn[5];
  double* qout[5];
  float2* sout;              // shadow of Q^(l) [3][Np] (null with rhs)
  long long Np;
  double* rhs;               // non-null: write RHS [5][N] instead of updating
  Scalars* sc;
  double alpha;
  int kchunk;
  int want_res;
  int want_rate;
};

// ---- TMA and mbarrier (inline PTX) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
// Request the shadow of plane k (padded plane k + 2) of this CTA's halo-2 box into a ring slot;
// the mbarrier completes when its BOX_BYTES have landed.  Called by one thread.
__device__ __forceinline__ void request_plane(const Args& A, Smem& sm, int slot, int x0, int y0, int k) {
  unsigned long long* b = &sm.bar[slot];
  // the slot's previous contents were read through the generic proxy before the last barrier
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(BOX_BYTES)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(&sm.sh[slot][0])),
      "l"(reinterpret_cast<unsigned long long>(&A.tm)), "r"(x0), "r"(y0), "r"(k + kG), "r"(0), "r"(smem_u32(b))
      : "memory");
}
// Wait for an mbarrier phase with a bounded number of polls; false if it never completed.
constexpr int kWaitPolls = 1 << 18;   // ~1 s on GB300 (each unanswered try_wait suspends a few microseconds)
__device__ __forceinline__ bool wait_bar(unsigned long long* bar, unsigned parity) {
  const unsigned b = smem_u32(bar);
  for (int it = 0; it < kWaitPolls; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ bool wait_slot(Smem& sm, int slot, unsigned parity) { return wait_bar(&sm.bar[slot], parity); }

// Plane k of the CTA starting at k0 - 2 uses ring slot ring(k) for the ((k - k0 + 2) / 4)-th time.
__device__ __forceinline__ unsigned plane_parity(int k, int k0) { return (unsigned)((k - k0 + 2) >> 2) & 1u; }

// 1/rho on the halo-2 points of a landed shadow plane (rho = rho' + 1).
__device__ __forceinline__ void inv_rho(Smem& sm, int slot) {
#pragma unroll
  for (int r = 0; r < NIR; ++r) {
    const int t = threadIdx.x + r * NT;
    if (t < NP2) sm.ir[slot][t] = f_rcp(sm.sh[slot][t].x + 1.f);
  }
}

// The three shadow pairs of an FP64 state node (the FP32 values the stage arithmetic uses).
__device__ __forceinline__ void shadow_of(const ConstsF& c, const double q[5], float2 out[NSH]) {
  const float rp = f64_to_f32(q[0] - 1.0);
  const float m1 = f64_to_f32(q[1]), m2 = f64_to_f32(q[2]), m3 = f64_to_f32(q[3]);
  const float ep = f64_to_f32(q[4] - c.e_inf);
  const float ir = f_rcp(rp + 1.f);
  const float pp = c.gm1 * (ep - 0.5f * ir * (m1 * m1 + m2 * m2 + m3 * m3));
  out[0] = make_float2(rp, ep);
  out[1] = make_float2(m1, m2);
  out[2] = make_float2(m3, pp);
}

// Metric record of one node (three 16-byte loads).
__device__ __forceinline__ void load_record(const float* M, long long p, float met[kMF]) {
  const float4* r = reinterpret_cast<const float4*>(M + p * kMF);
  const float4 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2);
  met[0] = a.x; met[1] = a.y; met[2] = a.z; met[3] = a.w;
  met[4] = b.x; met[5] = b.y; met[6] = b.z; met[7] = b.w;
  met[8] = c.x; met[9] = c.y; met[10] = c.z; met[11] = c.w;
}

// Metric record of this thread's halo-1 node of plane q (nb < 0: outside, zeros).
__device__ __forceinline__ void load_metrics(const Args& A, long long nb, int q, float met[kMF]) {
  if (nb < 0) {
#pragma unroll
    for (int f = 0; f < kMF; ++f) met[f] = 0.f;
    return;
  }
  load_record(A.M, nb + (long long)q * A.d.sk, met);
}

// A landed ring slot: the shadow pairs and 1/rho of its halo-2 points.
struct Plane {
  const float2* s;
  const float* ir;
};
__device__ __forceinline__ Plane plane(const Smem& sm, int slot) { return Plane{sm.sh[slot], sm.ir[slot]}; }
__device__ __forceinline__ float2 P_re(const Plane& P, int c) { return P.s[c]; }              // rho', e'
__device__ __forceinline__ float2 P_m12(const Plane& P, int c) { return P.s[NP2 + c]; }       // m1, m2
__device__ __forceinline__ float2 P_m3p(const Plane& P, int c) { return P.s[2 * NP2 + c]; }   // m3, p'
// The five conserved offsets (rho', m1, m2, m3, e') of a ring point: what the dissipation acts on.
__device__ __forceinline__ void load_q(const Plane& P, int c, float q[5]) {
  const float2 a = P_re(P, c), b = P_m12(P, c), d = P_m3p(P, c);
  q[0] = a.x; q[1] = b.x; q[2] = b.y; q[3] = d.x; q[4] = a.y;
}

// Nodal fluxes, spectral radii and sensors of one node of plane q (slots
// s_m, s_0, s_p of planes q-1, q, q+1) at halo-1 index t, into ring slot g.
__device__ void nodal(const Args& A, Smem& sm, long long nb, const float met[kMF], int s_m, int s_0, int s_p, int g) {
  const ConstsF& c = A.c;
  const int t = threadIdx.x;
  const int x1 = t % H1X, y1 = t / H1X;
  const bool tile = x1 >= 1 && x1 <= TX && y1 >= 1 && y1 <= TY;
  const int o = (y1 - 1) * TX + (x1 - 1);
  const int c2 = (y1 + 1) * H2X + (x1 + 1);
  float* Fx = &sm.fxy[g][0][0];
  float* Fz = &sm.fz[g][0][0];
  if (nb < 0) {
#pragma unroll 1
    for (int f = 0; f < NXF; ++f) Fx[f * NP1 + t] = 0.f;
    if (tile)
#pragma unroll 1
      for (int f = 0; f < NZF; ++f) Fz[f * NOUT + o] = 0.f;
    return;
  }
  float S[3][3];
#pragma unroll
  for (int dir = 0; dir < 3; ++dir)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) S[dir][cc] = met[3 * dir + cc];
  const float iV = met[MF_IV];
  const Plane P0 = plane(sm, s_0), Pm = plane(sm, s_m), Pp = plane(sm, s_p);
  // u, v, w, T at a node of the ring (plane P, halo-2 index cc)
  auto uvwT = [&](const Plane& P, int cc, float f[4]) {
    const float ir = P.ir[cc];
    const float2 a = P_m12(P, cc), b = P_m3p(P, cc);
    f[0] = a.x * ir;
    f[1] = a.y * ir;
    f[2] = b.x * ir;
    f[3] = c.gamma * (b.y + c.p_inf) * ir;
  };
  // gradients of u, v, w, T: L[n][j] = sum_dir (S^dir_j / (2V)) (f_{+} - f_{-})
  const float h = 0.5f * iV;
  float fxp[4], fxm[4], fyp[4], fym[4], fzp[4], fzm[4];
  uvwT(P0, c2 + 1, fxp);
  uvwT(P0, c2 - 1, fxm);
  uvwT(P0, c2 + H2X, fyp);
  uvwT(P0, c2 - H2X, fym);
  uvwT(Pp, c2, fzp);
  uvwT(Pm, c2, fzm);
  float L[4][3];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const float dx = fxp[n] - fxm[n], dy = fyp[n] - fym[n], dz = fzp[n] - fzm[n];
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) L[n][jj] = h * (S[0][jj] * dx + S[1][jj] * dy + S[2][jj] * dz);
  }
  const float2 re0 = P_re(P0, c2), m12 = P_m12(P0, c2), m3p = P_m3p(P0, c2);
  const float rho = re0.x + 1.f;
  const float m1 = m12.x, m2 = m12.y, m3 = m3p.x;
  float f0[4];
  uvwT(P0, c2, f0);
  const float u = f0[0], v = f0[1], w = f0[2], T = f0[3];
  const float pp = m3p.y;
  const float ep = re0.y;
  const float a = f_sqrt(T);
  const float mu = c.mu_ref * (T * a) * c.sut_num * f_rcp(T + c.S_hat);
  // strain rate (symmetric), eddy viscosity, stresses
  const float s11 = L[0][0], s22 = L[1][1], s33 = L[2][2];
  const float s12 = 0.5f * (L[0][1] + L[1][0]), s13 = 0.5f * (L[0][2] + L[2][0]), s23 = 0.5f * (L[1][2] + L[2][1]);
  const float div = s11 + s22 + s33;
  const float SS = s11 * s11 + s22 * s22 + s33 * s33 + 2.f * (s12 * s12 + s13 * s13 + s23 * s23);
  const float Smod = f_sqrt(2.f * SS);
  const float csd = c.C_s * met[MF_D];
  const float mu_sgs = rho * (csd * csd) * Smod;
  const float m2e = 2.f * (mu + mu_sgs);
  const float k_eff = mu * c.k_lam + mu_sgs * c.k_sgs;
  const float d3 = div * (1.f / 3.f);
  const float t11 = m2e * (s11 - d3), t22 = m2e * (s22 - d3), t33 = m2e * (s33 - d3);
  const float t12 = m2e * s12, t13 = m2e * s13, t23 = m2e * s23;
  // Cartesian viscous fluxes F_x, F_y, F_z (momentum x, y, z; energy)
  const float F[3][4] = {{t11, t12, t13, u * t11 + v * t12 + w * t13 + k_eff * L[3][0]},
                         {t12, t22, t23, u * t12 + v * t22 + w * t23 + k_eff * L[3][1]},
                         {t13, t23, t33, u * t13 + v * t23 + w * t33 + k_eff * L[3][2]}};
  const float h0 = ep + pp + c.ep_inf;   // e + p
  float lam[3], H[3][5];
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    const float U = S[dir][0] * u + S[dir][1] * v + S[dir][2] * w;
    const float smag = f_sqrt(S[dir][0] * S[dir][0] + S[dir][1] * S[dir][1] + S[dir][2] * S[dir][2]);
    lam[dir] = fabsf(U) + a * smag;
    H[dir][0] = rho * U;
    H[dir][1] = m1 * U + pp * S[dir][0] - (S[dir][0] * F[0][0] + S[dir][1] * F[1][0] + S[dir][2] * F[2][0]);
    H[dir][2] = m2 * U + pp * S[dir][1] - (S[dir][0] * F[0][1] + S[dir][1] * F[1][1] + S[dir][2] * F[2][1]);
    H[dir][3] = m3 * U + pp * S[dir][2] - (S[dir][0] * F[0][2] + S[dir][1] * F[1][2] + S[dir][2] * F[2][2]);
    H[dir][4] = h0 * U - (S[dir][0] * F[0][3] + S[dir][1] * F[1][3] + S[dir][2] * F[2][3]);
  }
  const float r0 = cbrt_pos(lam[0]), r1 = cbrt_pos(lam[1]), r2 = cbrt_pos(lam[2]);
  // pressure sensors (p' = p - p_inf; denominators add 4 p_inf back)
  const float pxm = P_m3p(P0, c2 - 1).y, pxp = P_m3p(P0, c2 + 1).y;
  const float pym = P_m3p(P0, c2 - H2X).y, pyp = P_m3p(P0, c2 + H2X).y;
  const float pzm = P_m3p(Pm, c2).y, pzp = P_m3p(Pp, c2).y;
  const float p4 = 4.f * c.p_inf;
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    Fx[(X_HX + m) * NP1 + t] = H[0][m];
    Fx[(X_HY + m) * NP1 + t] = H[1][m];
  }
  Fx[X_LX * NP1 + t] = lam[0] + r0 * (r1 * r1 + r2 * r2);
  Fx[X_LY * NP1 + t] = lam[1] + r1 * (r0 * r0 + r2 * r2);
  Fx[X_NX * NP1 + t] = fabsf(pxp - 2.f * pp + pxm) * f_rcp(pxp + 2.f * pp + pxm + p4);
  Fx[X_NY * NP1 + t] = fabsf(pyp - 2.f * pp + pym) * f_rcp(pyp + 2.f * pp + pym + p4);
  if (tile) {
#pragma unroll
    for (int m = 0; m < 5; ++m) Fz[(Z_HZ + m) * NOUT + o] = H[2][m];
    Fz[Z_L * NOUT + o] = lam[2] + r2 * (r0 * r0 + r1 * r1);
    Fz[Z_N * NOUT + o] = fabsf(pzp - 2.f * pp + pzm) * f_rcp(pzp + 2.f * pp + pzm + p4);
    Fz[Z_IV * NOUT + o] = iV;
  }
}

// The xi and eta dissipation faces of one plane (ring slots: prim s_0, fluxes g),
// each computed once by one thread.  Tasks are laid out one 32-lane row per
// face row so that a warp touches one shared-memory row (no bank conflicts).
constexpr int NTX = 32 * TY, NTY = 32 * (TY + 1);
static_assert(TX + 1 <= 32, "xi face row fits a warp");

__device__ void plane_faces(const Args& A, Smem& sm, int s_0, int g) {
  const Plane P = plane(sm, s_0);
  const float* Fx = &sm.fxy[g][0][0];
  for (int task = threadIdx.x; task < NTX + NTY; task += NT) {
    float qm[5], q0[5], q1[5], q2[5], out[5];
    if (task < NTX) {
      const int oy = task >> 5, fx = task & 31;
      if (fx > TX) continue;
      const int e = oy * (TX + 1) + fx;
      const int a = (oy + 1) * H1X + fx;           // halo-1 index of the left node
      const int cq = (oy + 2) * H2X + fx + 1;      // halo-2 index of the left node
      load_q(P, cq - 1, qm);
      load_q(P, cq, q0);
      load_q(P, cq + 1, q1);
      load_q(P, cq + 2, q2);
      face_flux(A.c, Fx[X_LX * NP1 + a], Fx[X_LX * NP1 + a + 1], Fx[X_NX * NP1 + a], Fx[X_NX * NP1 + a + 1],
                qm, q0, q1, q2, out);
#pragma unroll
      for (int m = 0; m < 5; ++m) sm.dx[m][e] = out[m];
    } else {
      const int fy = (task - NTX) >> 5, ox = (task - NTX) & 31;
      if (ox >= TX) continue;
      const int e2 = fy * TX + ox;
      const int a = fy * H1X + ox + 1;             // halo-1 index of the lower node
      const int cq = (fy + 1) * H2X + ox + 2;      // halo-2 index of the lower node
      load_q(P, cq - H2X, qm);
      load_q(P, cq, q0);
      load_q(P, cq + H2X, q1);
      load_q(P, cq + 2 * H2X, q2);
      face_flux(A.c, Fx[X_LY * NP1 + a], Fx[X_LY * NP1 + a + H1X], Fx[X_NY * NP1 + a], Fx[X_NY * NP1 + a + H1X],
                qm, q0, q1, q2, out);
#pragma unroll
      for (int m = 0; m < 5; ++m) sm.dy[m][e2] = out[m];
    }
  }
}


constexpr int kMinBlocks = NT <= 320 ? 2 : 1;

__global__ void __launch_bounds__(NT, kMinBlocks) k_fused32(const __grid_constant__ Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // TMA destinations need 128-byte alignment; the launch adds 128 bytes of room for it
  Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  const Dims& d = A.d;
  const ConstsF& c = A.c;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * A.kchunk;
  const int k1 = min(k0 + A.kchunk, d.nk);          // output planes [k0, k1)
  const int t = threadIdx.x;
  const int ox = t & 31, oy = t >> 5;
  const bool outth = t < NOT && ox < TX;
  const int o = oy * TX + ox;                       // tile index of the output node
  const int oi = i0 + ox, oj = j0 + oy;
  const bool outv = outth && oi < d.ni && oj < d.nj;
  const bool adv = outv && (d.topo != JZ_TOPO_JET || (oi >= 1 && oi <= d.ni - 2 && oj >= 1 && oj <= d.nj - 2));
  const int c1 = (oy + 1) * H1X + (ox + 1);
  const int c2 = (oy + 2) * H2X + (ox + 2);
  // the halo-2 box starts at real (i0 - 2, j0 - 2): padded (i0, j0); x0 * 8 bytes is a multiple
  // of 16 because TX is even
  const int x0 = i0, y0 = j0;

  long long nb;                                    // halo-1 node of this thread (nodal work)
  {
    const int i = i0 - 1 + t % H1X, j = j0 - 1 + t / H1X;
    nb = in_padded(d, i, j) ? pidx(d, i, j, 0) : -1;
  }
  const long long ob = outv ? pidx(d, oi, oj, 0) : 0;   // output node
  // prime: mbarriers, then planes k0-2 .. k0 requested; k0-2 and k0-1 waited for
  int last_req = k0 - 3;                           // thread 0: last plane requested
  if (t == 0) {
    for (int s = 0; s < NRING; ++s) bar_init(&sm.bar[s], 1);
    sm.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0) {
    for (int q = k0 - 2; q <= k0; ++q) request_plane(A, sm, ring(q), x0, y0, q);
    last_req = k0;
  }
  for (int q = k0 - 2; q <= k0 - 1; ++q) {
    if (!wait_slot(sm, ring(q), plane_parity(q, k0))) sm.fail = q + 1000000;
    inv_rho(sm, ring(q));
  }

  float Hz_prev[5] = {0, 0, 0, 0, 0};   // H^zeta(p-1)
  float Dz_prev[5] = {0, 0, 0, 0, 0};   // d^zeta(p-1/2)
  float Qz_prev[5] = {0, 0, 0, 0, 0};   // Q(p-1), FP32
  float Lz = 0.f, Nz = 0.f;             // Lambda^zeta(p), nu^zeta(p)
  const float adt = f64_to_f32(A.alpha * A.sc->dt);
  float res = 0.f, rate = 0.f;

  for (int p = k0 - 2; p < k1; ++p) {
    // (a) metrics of plane p+1 (used in (b)); the shadow of plane p+2 (requested one plane
    // earlier) and its 1/rho
    float met[kMF];
    load_metrics(A, nb, p + 1, met);
    // L2 hints one plane ahead: metrics of plane p+2 (next iteration's nodal work)
    // and Q^n of plane p+1 (next iteration's update)
    if (nb >= 0 && p + 2 <= k1) {
      // a 48-byte record spans two 32-byte sectors; with the neighbours' requests every
      // sector of the row is asked for
      const float* pm = A.M + (nb + (long long)(p + 2) * d.sk) * kMF;
      prefetch_l2(pm);
      prefetch_l2(pm + 8);
    }
    if (adv && !A.rhs && p + 1 < k1) {
      const long long pq = ob + (long long)(p + 1) * d.sk;
#pragma unroll
      for (int m = 0; m < 5; ++m) prefetch_l2(A.qn[m] + pq);
    }
    // after a wait ran out no plane is requested or waited for any more (the CTA finishes on
    // stale data and the host reports the error)
    if (sm.fail == 0 && !wait_slot(sm, ring(p + 2), plane_parity(p + 2, k0))) sm.fail = p + 2 + 1000000;
    inv_rho(sm, ring(p + 2));
    __syncthreads();
    // the slot of plane p-1 is free: request plane p+3 into it
    if (t == 0 && p + 3 <= k1 + 1 && sm.fail == 0) {
      request_plane(A, sm, ring(p + 3), x0, y0, p + 3);
      last_req = p + 3;
    }
    // (b) nodal quantities of plane p+1, then the xi/eta faces of plane p
    nodal(A, sm, nb, met, ring(p), ring(p + 1), ring(p + 2), (p + 1) & 1);
    plane_faces(A, sm, ring(p), p & 1);
    __syncthreads();
    // (c) zeta face p+1/2 and the output plane p
    if (outth) {
      const float* Z0 = &sm.fz[p & 1][0][0];
      const float* Z1 = &sm.fz[(p + 1) & 1][0][0];
      const Plane P0 = plane(sm, ring(p)), P1 = plane(sm, ring(p + 1)), P2 = plane(sm, ring(p + 2));
      const float Lz1 = Z1[Z_L * NOUT + o], Nz1 = Z1[Z_N * NOUT + o];
      // Q^n of this output node, requested before the zeta-face work that hides its latency
      double qn_r[5];
      const long long pp = ob + (long long)p * d.sk;
      if (p >= k0 && adv && !A.rhs) {
#pragma unroll
        for (int m = 0; m < 5; ++m) qn_r[m] = __ldg(A.qn[m] + pp);
      }
      float q0[5], q1[5], q2[5], Dz[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      load_q(P0, c2, q0);
      load_q(P1, c2, q1);
      load_q(P2, c2, q2);
      if (p >= k0 - 1) face_flux(c, Lz, Lz1, Nz, Nz1, Qz_prev, q0, q1, q2, Dz);
      if (p >= k0 && outv) {
        const float* F0 = &sm.fxy[p & 1][0][0];
        const int ex = oy * (TX + 1) + ox, ey = oy * TX + ox;
        const float iV = Z0[Z_IV * NOUT + o];
        float R[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          float acc = 0.5f * (F0[(X_HX + m) * NP1 + c1 + 1] - F0[(X_HX + m) * NP1 + c1 - 1]) -
                      (sm.dx[m][ex + 1] - sm.dx[m][ex]);
          acc += 0.5f * (F0[(X_HY + m) * NP1 + c1 + H1X] - F0[(X_HY + m) * NP1 + c1 - H1X]) -
                 (sm.dy[m][ey + TX] - sm.dy[m][ey]);
          acc += 0.5f * (Z1[(Z_HZ + m) * NOUT + o] - Hz_prev[m]) - (Dz[m] - Dz_prev[m]);
          R[m] = acc * iV;
        }
        if (A.rhs) {
          const long long N = (long long)d.ni * d.nj * d.nk;
          const long long ridx = ((long long)p * d.nj + oj) * d.ni + oi;
#pragma unroll
          for (int m = 0; m < 5; ++m) A.rhs[m * N + ridx] = adv ? f32_to_f64(R[m]) : 0.0;
        } else if (adv) {
          double qnew[5];
#pragma unroll
          for (int m = 0; m < 5; ++m) {
            qnew[m] = qn_r[m] - f32_to_f64(adt * R[m]);
            A.qout[m][pp] = qnew[m];
          }
          float2 shn[NSH];
          shadow_of(c, qnew, shn);
#pragma unroll
          for (int m = 0; m < NSH; ++m) A.sout[m * A.Np + pp] = shn[m];
          if (A.want_rate) {
            const float rho = f64_to_f32(qnew[0]);
            const float ir = f_rcp(rho);
            const float m1 = f64_to_f32(qnew[1]), m2 = f64_to_f32(qnew[2]), m3 = f64_to_f32(qnew[3]);
            const float u = m1 * ir, v = m2 * ir, w = m3 * ir;
            const float pr = c.gm1 * (f64_to_f32(qnew[4] - c.e_inf) - 0.5f * (m1 * u + m2 * v + m3 * w)) + c.p_inf;
            const float a = f_sqrt(c.gamma * pr * ir);
            float ls = 0.f;            float mr[kMF];
            load_record(A.M, pp, mr);
#pragma unroll
            for (int dir = 0; dir < 3; ++dir) {
              const float sx = mr[3 * dir], sy = mr[3 * dir + 1], sz = mr[3 * dir + 2];
              ls += fabsf(sx * u + sy * v + sz * w) + a * f_sqrt(sx * sx + sy * sy + sz * sz);
            }
            rate = fmaxf(rate, ls * iV);
          }
        } else {
#pragma unroll
          for (int m = 0; m < 5; ++m) A.qout[m][pp] = A.qin[m][pp];
          A.sout[pp] = P_re(P0, c2);
          A.sout[A.Np + pp] = P_m12(P0, c2);
          A.sout[2 * A.Np + pp] = P_m3p(P0, c2);
        }
        if (adv) res += R[0] * R[0];
      }
      // rotate the zeta registers
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        Hz_prev[m] = Z0[(Z_HZ + m) * NOUT + o];
        Dz_prev[m] = Dz[m];
        Qz_prev[m] = q0[m];
      }
      Lz = Lz1;
      Nz = Nz1;
    }
    // no barrier here: the next iteration's phase (a) writes 1/rho of ring slot p+3, which no
    // thread reads in this iteration; the barrier after it orders the flux rings.
  }
  if (t == 0 && sm.fail != 0) {
    // a wait ran out: give the copies still in flight a bounded time to land before the CTA's
    // shared memory is released, then report
    for (int q = sm.fail - 1000000; q <= last_req; ++q) wait_slot(sm, ring(q), plane_parity(q, k0));
    atomicOr(&A.sc->wait_timeout, 1);
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


// FP32 shadow of the FP64 state on every padded node (full) or on the shell that the boundary
// conditions and the ghost fill rewrite: i in {-2, -1, 0, ni-1, ni, ni+1} (all j, k), then j in
// {-2, -1, 0, nj-1, nj, nj+1} and k in {-2, -1, nk, nk+1} over the remaining nodes.
__global__ void k_shadow(Dims d, ConstsF c, State q, int full) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, k;
  if (full) {
    const Box b{-kG, -kG, -kG, d.ni + 2 * kG, d.nj + 2 * kG, d.nk + 2 * kG};
    if (!box_coord(b, t, i, j, k)) return;
  } else {
    const int ii = max(d.ni - 2, 0), ij = max(d.nj - 2, 0);
    const long long cI = 6LL * (d.nj + 2 * kG) * (d.nk + 2 * kG);
    const long long cJ = 6LL * ii * (d.nk + 2 * kG);
    const long long cK = 4LL * ii * ij;
    int a;
    if (t < cI) {
      a = (int)(t % 6);
      const long long r = t / 6;
      j = (int)(r % (d.nj + 2 * kG)) - kG;
      k = (int)(r / (d.nj + 2 * kG)) - kG;
      i = a < 3 ? a - kG : d.ni - 1 + (a - 3);
    } else if ((t -= cI) < cJ) {
      a = (int)(t % 6);
      const long long r = t / 6;
      i = 1 + (int)(r % ii);
      k = (int)(r / ii) - kG;
      j = a < 3 ? a - kG : d.nj - 1 + (a - 3);
    } else if ((t -= cJ) < cK) {
      a = (int)(t % 4);
      const long long r = t / 4;
      i = 1 + (int)(r % ii);
      j = 1 + (int)(r / ii);
      k = a < 2 ? a - kG : d.nk + (a - 2);
    } else {
      return;
    }
  }
  const long long p = pidx(d, i, j, k);
  double v[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) v[m] = q.q[m][p];
  float2 s[NSH];
  shadow_of(c, v, s);
#pragma unroll
  for (int m = 0; m < NSH; ++m) q.sh[m * d.Np + p] = s[m];
}

// Self-check of the bounded wait: one warp initialises an mbarrier that nothing ever arrives at
// and waits for it with the stage kernel's bounded poll; the wait must run out and return.
__global__ void k_wait_check(int* timed_out, long long* cycles) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    bar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long long t0 = clock64();
  const bool ok = wait_bar(&bar, 0);
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    *timed_out = ok ? 0 : 1;
    *cycles = t1 - t0;
  }
}

ConstsF make_constsf(const Consts& c) {
  ConstsF f;
  f.gamma = (float)c.gamma; f.gm1 = (float)c.gm1; f.mu_ref = (float)c.mu_ref; f.S_hat = (float)c.S_hat;
  f.sut_num = (float)c.sut_num; f.k_lam = (float)c.k_lam; f.k_sgs = (float)c.k_sgs; f.C_s = (float)c.C_s;
  f.kappa2 = (float)c.kappa2; f.kappa4 = (float)c.kappa4; f.p_inf = (float)c.p_inf;
  f.e_inf = c.p_inf / c.gm1;
  f.ep_inf = (float)(f.e_inf + c.p_inf);
  return f;
}

constexpr int kSmemBytes = (int)sizeof(Smem) + 128;    // + room to align the ring to 128 bytes
static_assert(TX % 2 == 0, "the TMA box must start on a 16-byte boundary (x0 = i0 padded, 8-byte elements)");

// The dynamic shared-memory size above 48 KB must be allowed once per device.
cudaError_t allow_smem() {
  static bool attr[64] = {false};
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return e0;
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_fused32, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  return cudaSuccess;
}

}  // namespace

// Resident CTAs of the fused kernel on the whole device (SMs x CTAs per SM).
cudaError_t fused32_slots(int* slots) {
  cudaError_t e = allow_smem();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused32, NT, kSmemBytes);
  if (e != cudaSuccess) return e;
  *slots = sms * (per > 0 ? per : 1);
  return cudaSuccess;
}

cudaError_t make_shadow_map(const Dims& d, float2* sh, void* tmap128) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorInvalidValue;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // 8-byte elements (one float2 pair each); rows of Pi, planes of Pi x Pj, three arrays of Np
  const cuuint64_t dims[4] = {(cuuint64_t)d.Pi, (cuuint64_t)d.Pj, (cuuint64_t)d.Pk, (cuuint64_t)NSH};
  const cuuint64_t strides[3] = {(cuuint64_t)d.Pi * 8, (cuuint64_t)d.sk * 8, (cuuint64_t)d.Np * 8};
  const cuuint32_t box[4] = {(cuuint32_t)H2X, (cuuint32_t)H2Y, 1, (cuuint32_t)NSH};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(tmap128), CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, sh, dims, strides,
                            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t shadow_refresh(const Dims& d, const Consts& c, const State& q, int full, cudaStream_t st) {
  long long n;
  if (full) {
    n = (long long)(d.ni + 2 * kG) * (d.nj + 2 * kG) * (d.nk + 2 * kG);
  } else {
    const long long ii = std::max(d.ni - 2, 0), ij = std::max(d.nj - 2, 0);
    n = 6LL * (d.nj + 2 * kG) * (d.nk + 2 * kG) + 6LL * ii * (d.nk + 2 * kG) + 4LL * ii * ij;
  }
  k_shadow<<<blocks_for(n, 256), 256, 0, st>>>(d, make_constsf(c), q, full);
  return cudaGetLastError();
}

cudaError_t fused32(const Dims& d, const Consts& c, const float* Mf, const State& qin, const void* tm_in,
                    const State& qn, const State& qout, Scalars* sc, double alpha, int want_res, int want_rate,
                    double* rhs_flat, int kchunk, cudaStream_t st) {
  cudaError_t e0 = allow_smem();
  if (e0 != cudaSuccess) return e0;
  Args A;
  std::memcpy(&A.tm, tm_in, sizeof(CUtensorMap));
  A.d = d;
  A.c = make_constsf(c);
  A.M = Mf;
  for (int m = 0; m < 5; ++m) {
    A.qin[m] = qin.q[m];
    A.qn[m] = qn.q[m];
    A.qout[m] = qout.q[m];
  }
  A.sout = qout.sh;
  A.Np = d.Np;
  A.rhs = rhs_flat;
  A.sc = sc;
  A.alpha = alpha;
  A.kchunk = kchunk > 0 ? kchunk : d.nk;
  A.want_res = want_res;
  A.want_rate = want_rate;
  dim3 grid((d.ni + TX - 1) / TX, (d.nj + TY - 1) / TY, (d.nk + A.kchunk - 1) / A.kchunk);
  k_fused32<<<grid, NT, kSmemBytes, st>>>(A);
  return cudaGetLastError();
}

cudaError_t wait_check(int* dev_timed_out, long long* dev_cycles, cudaStream_t st) {
  k_wait_check<<<1, 32, 0, st>>>(dev_timed_out, dev_cycles);
  return cudaGetLastError();
}

int fused32_tile_x() { return TX; }
int fused32_tile_y() { return TY; }

}  // namespace jz
