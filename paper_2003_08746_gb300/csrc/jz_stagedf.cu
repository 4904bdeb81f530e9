// Pair form of the FP64 stage: the work of the four passes of jz_stage64.cu (nodal, viscous,
// faces, update; Algorithm 2's inviscid flux, dissipation, viscous flux, RHS and
// Update(Cons, alpha_l)) in three kernels, with every flux, dissipation and SGS operation in
// double-float arithmetic (jz_df.cuh: pairs of FP32 numbers, ~48 significant bits) and the stage
// combination Q^n - alpha dt RHS in FP64.  The state stays FP64; the nodal pass reads it once and
// leaves a double-float copy for the dissipation; the intermediate fields are double-float pairs
// (float2) in the FP64 form's work arrays (same size); the metrics are a double-float copy made
// when the solver is created.  The last kernel forms the face fluxes and sums them into the RHS
// of each node without storing them, so the pair form's results are those of separate faces and
// update passes bit for bit.
//
// The nodal and viscous passes are launched on 3-D grids (64 x 4 threads per block along i and j,
// one block row per k), so no pass divides a flat index.
#include "jz_dfconsts.cuh"

namespace jz {
namespace {

constexpr int BX = 64, BY = 4;

// node of a 3-D launch over the box [i0, i0 + ei) x [j0, j0 + ej) x [k0, k0 + ek)
__device__ __forceinline__ bool node3(int i0, int j0, int k0, int ei, int ej, int& i, int& j, int& k) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= ei || y >= ej) return false;
  i = i0 + x;
  j = j0 + y;
  k = k0 + (int)blockIdx.z;
  return true;
}

__device__ __forceinline__ bool advanced(const Dims& d, int i, int j) {
  return d.topo != JZ_TOPO_JET || (i >= 1 && i <= d.ni - 2 && j >= 1 && j <= d.nj - 2);
}


// A: every padded node.  Primitives, Sutherland mu, spectral radii and their anisotropic
// scaling; the double-float copy of Q for the viscous and faces passes; at stage 1 also the CFL
// rate of Q^n (block max, one atomic per block).
// Five blocks per SM (48 registers): the pass is bound by DRAM traffic and gains from the extra
// warps (11.3 against 12.8 ms per launch on 1000 x 400 x 500); the viscous pass loses from the same.
__global__ void __launch_bounds__(BX* BY, 5) k_nodal_df(Dims d, ConstsDF c, DFMetrics M, Work64 w, State q,
                                                     QDF qdf, double* rate_max) {
  int i, j, k;
  double rate = 0.0;
  if (node3(-kG, -kG, -kG, d.ni + 2 * kG, d.nj + 2 * kG, i, j, k)) {
    const long long p = pidx(d, i, j, k);
    const dfl rho = df_of(q.q[0][p]), m1 = df_of(q.q[1][p]), m2 = df_of(q.q[2][p]), m3 = df_of(q.q[3][p]),
              e = df_of(q.q[4][p]);
    st(qdf.q[0], p, rho); st(qdf.q[1], p, m1); st(qdf.q[2], p, m2); st(qdf.q[3], p, m3); st(qdf.q[4], p, e);
    const dfl ir = df_rcp(rho);
    const dfl u = df_mul(m1, ir), v = df_mul(m2, ir), ww = df_mul(m3, ir);
    const dfl ke = df_fma(m3, ww, df_fma(m2, v, df_mul(m1, u)));            // rho |u|^2
    const dfl pr = df_sub(df_mul(e, c.gm1), df_mul(ke, c.gm1_half));    // (gamma-1)(e - rho|u|^2/2)
    const dfl T = df_mul(df_mul(pr, c.gamma), ir);
    const dfl a = df_sqrt(T);
    // Sutherland, eq. (sutherland), with T_inf = 1
    const dfl mu = df_mul(df_mul(c.mu_sut, df_mul(T, a)), df_rcp(df_add(T, c.S_hat)));
    st(w.u, p, u); st(w.v, p, v); st(w.w, p, ww); st(w.T, p, T); st(w.p, p, pr); st(w.mu, p, mu);
    dfl lam[3];
    for (int dir = 0; dir < 3; ++dir) {
      const dfl sx = df_load(M.S[3 * dir], p), sy = df_load(M.S[3 * dir + 1], p), sz = df_load(M.S[3 * dir + 2], p);
      const dfl U = df_fma(sz, ww, df_fma(sy, v, df_mul(sx, u)));
      lam[dir] = df_fma(a, df_load(M.Smag[dir], p), df_abs(U));
    }
    if (rate_max && i >= 0 && i < d.ni && j >= 0 && j < d.nj && k >= 0 && k < d.nk && advanced(d, i, j))
      rate = df_to_f64(df_mul(df_add(df_add(lam[0], lam[1]), lam[2]), df_load(M.invV, p)));
    dfl Lam[3];
    aniso_df(c, lam, Lam);
    st(w.Lam[0], p, Lam[0]); st(w.Lam[1], p, Lam[1]); st(w.Lam[2], p, Lam[2]);
  }
  if (rate_max) {
    // block max -> one atomic per block (non-negative doubles order like their bits)
    __shared__ double redm[BX * BY / 32];
    const int tid = threadIdx.y * BX + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    if ((tid & 31) == 0) redm[tid >> 5] = rate;
    __syncthreads();
    if (tid < 32) {
      double x = tid < BX * BY / 32 ? redm[tid] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
      if (tid == 0 && x > 0.0)
        atomicMax(reinterpret_cast<unsigned long long*>(rate_max), (unsigned long long)__double_as_longlong(x));
    }
  }
}

// B: nodes within one layer of the real region (the nodes whose fluxes the faces read).
// Gradients by the chain rule, strain rate, Smagorinsky eddy viscosity, stresses and heat flux;
// the transformed flux H^dir = E^dir - S^dir_j F_j, inviscid part E^dir from the nodal
// primitives and the pair copy of Q, written once; pressure sensors.  Forming E^dir here rather
// than in the nodal pass saves its store there and the load of it here (160 bytes per node):
// 17.1 against 20.2 + 3.2 ms per launch on 1000 x 400 x 500.  Four blocks per SM (64 registers,
// a few spilled): 17.1 against 17.6 ms at 80 registers.  Unnormalized sums and products inside
// each chain (normalized before stores, roots and reciprocals; jz_df.cuh): 15.2 against 17.1 ms,
// ~20% fewer FP32 operations; residuals move by up to 5e-13 of their norm, states by 2e-15.
__global__ void __launch_bounds__(BX* BY, 4) k_viscous_df(Dims d, ConstsDF c, DFMetrics M, Work64 w, QDF qdf) {
  int i, j, k;
  if (!node3(-1, -1, -1, d.ni + 2, d.nj + 2, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const long long s[3] = {1, d.sj, d.sk};
  const double* f[4] = {w.u, w.v, w.w, w.T};
  dfl S[3][3];
  for (int dir = 0; dir < 3; ++dir)
    for (int cc = 0; cc < 3; ++cc) S[dir][cc] = df_load(M.S[3 * dir + cc], p);
  const dfl iV = df_load(M.invV, p);
  // G[n][j] = sum_dir S^dir_j (f_n[+dir] - f_n[-dir]); the gradient is h G with h = 1/(2V)
  dfl G[4][3];
  for (int n = 0; n < 4; ++n) {
    dfl dd[3];
    for (int dir = 0; dir < 3; ++dir) dd[dir] = df_sub_l(ld(f[n], p + s[dir]), ld(f[n], p - s[dir]));
    for (int jj = 0; jj < 3; ++jj)
      G[n][jj] = df_n(df_fma_l(S[2][jj], dd[2], df_fma_l(S[1][jj], dd[1], df_mul_l(S[0][jj], dd[0]))));
  }
  const dfl h = df_scale(iV, 0.5f);
  // |S| = h sqrt(2 sum G_ii^2 + sum_{i<j} A_ij^2), A_ij = G_ij + G_ji
  const dfl A12 = df_add_l(G[0][1], G[1][0]), A13 = df_add_l(G[0][2], G[2][0]), A23 = df_add_l(G[1][2], G[2][1]);
  const dfl Gd = df_add_l(df_add_l(G[0][0], G[1][1]), G[2][2]);
  const dfl DG = df_fma_l(G[2][2], G[2][2], df_fma_l(G[1][1], G[1][1], df_mul_l(G[0][0], G[0][0])));
  const dfl AA = df_fma_l(A23, A23, df_fma_l(A13, A13, df_mul_l(A12, A12)));
  const dfl mu = ld(w.mu, p);
  const dfl csd = df_mul_l(df_load(M.Delta, p), c.C_s);
  // Smagorinsky eddy viscosity rho (C_s Delta)^2 |S|
  const dfl rho = ld(qdf.q[0], p);
  const dfl mu_sgs = df_n(df_mul_l(df_mul_l(rho, df_mul_l(csd, csd)),
                                   df_mul_l(h, df_sqrt(df_n(df_add_l(df_scale(DG, 2.f), AA))))));
  const dfl mt = df_add_l(mu, mu_sgs);
  const dfl mV = df_mul_l(mt, iV), mh = df_mul_l(mt, h);
  const dfl kh = df_mul_l(df_add_l(df_mul_l(mu, c.k_lam), df_mul_l(mu_sgs, c.k_sgs)), h);   // k_eff h
  const dfl d3 = df_mul_l(Gd, c.third);                                                       // Gd / 3
  const dfl t11 = df_mul_l(mV, df_sub_l(G[0][0], d3)), t22 = df_mul_l(mV, df_sub_l(G[1][1], d3)),
            t33 = df_mul_l(mV, df_sub_l(G[2][2], d3));
  const dfl t12 = df_mul_l(mh, A12), t13 = df_mul_l(mh, A13), t23 = df_mul_l(mh, A23);
  const dfl tau[3][3] = {{t11, t12, t13}, {t12, t22, t23}, {t13, t23, t33}};
  const dfl vel[3] = {ld(w.u, p), ld(w.v, p), ld(w.w, p)};
  dfl F[3][4];
  for (int jj = 0; jj < 3; ++jj) {
    F[jj][0] = tau[0][jj];
    F[jj][1] = tau[1][jj];
    F[jj][2] = tau[2][jj];
    F[jj][3] = df_fma_l(kh, G[3][jj],
                        df_fma_l(vel[2], tau[2][jj], df_fma_l(vel[1], tau[1][jj], df_mul_l(vel[0], tau[0][jj]))));
  }
  const dfl pc = ld(w.p, p);
  const dfl mq[3] = {ld(qdf.q[1], p), ld(qdf.q[2], p), ld(qdf.q[3], p)};
  const dfl h0 = df_add_l(ld(qdf.q[4], p), pc);                                               // e + p
  for (int dir = 0; dir < 3; ++dir) {
    const dfl U = df_fma_l(S[dir][2], vel[2], df_fma_l(S[dir][1], vel[1], df_mul_l(S[dir][0], vel[0])));
    dfl E[5];
    E[0] = df_mul_l(rho, U);
    for (int jj = 0; jj < 3; ++jj) E[jj + 1] = df_fma_l(mq[jj], U, df_mul_l(pc, S[dir][jj]));
    E[4] = df_mul_l(h0, U);
    st(w.H[dir][0], p, df_n(E[0]));
    for (int m = 0; m < 4; ++m) {
      const dfl sf = df_fma_l(S[dir][2], F[2][m], df_fma_l(S[dir][1], F[1][m], df_mul_l(S[dir][0], F[0][m])));
      st(w.H[dir][m + 1], p, df_n(df_sub_l(E[m + 1], sf)));
    }
  }
  // pressure sensor along each direction: |p+ - 2p + p-| / (p+ + 2p + p-)
  const dfl pc2 = df_scale(pc, 2.f);
  for (int dir = 0; dir < 3; ++dir) {
    const dfl sum = df_add_l(ld(w.p, p + s[dir]), ld(w.p, p - s[dir]));
    st(w.nu[dir], p, df_n(df_mul_l(df_abs(df_n(df_sub_l(sum, pc2))), df_rcp(df_n(df_add_l(sum, pc2))))));
  }
}

// C + D: Turkel-Vatsa dissipation combined with the face sum of H into the doubled total face
// flux G = H_n + H_(n+1) - 2 d_(n+1/2), and, in the same kernel, 2 V RHS = sum_dir (G(p) -
// G(p - s_dir)) in double-float with the stage combination Q^n - alpha dt RHS in FP64 (mode 0)
// or the RHS itself (mode 1).  The face fluxes never leave the SM: a block of 32 x 16 threads
// marches along k over a chunk of planes; the thread at (i, j) forms the three faces i + 1/2,
// j + 1/2, k + 1/2 of its node, takes the face i - 1/2 from the lane below it (shuffle), the face
// j - 1/2 from the row below it (shared memory) and the face k - 1/2 from its own previous plane.
// Column 0 and row 0 of the block are that halo (31 x 15 nodes updated per block and plane).
constexpr int FX = 32, FY = 16;

template <int DIR>
__device__ __forceinline__ void face_df(const ConstsDF& c, const Work64& w, const QDF& qdf, long long p,
                                        long long sd, dfl G[5]) {
  const dfl eps2 = df_mul(df_max(ld(w.nu[DIR], p), ld(w.nu[DIR], p + sd)), c.kappa2);
  const dfl k4 = df_sub(c.kappa4, eps2);
  const dfl eps4 = df_gt0(k4) ? k4 : df_make(0.f, 0.f);
  // 2 d = a32 d1 - b2 e3 with Ls = 2 L_f, b2 = Ls eps4, a32 = 3 b2 + Ls eps2
  const dfl Ls = df_add(ld(w.Lam[DIR], p), ld(w.Lam[DIR], p + sd));
  const dfl b2 = df_mul(Ls, eps4);
  const dfl a32 = df_fma(Ls, eps2, df_mul_f(b2, 3.f));
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const double* Q = qdf.q[m];
    const dfl d1 = df_sub(ld(Q, p + sd), ld(Q, p));
    const dfl e3 = df_sub(ld(Q, p + 2 * sd), ld(Q, p - sd));
    const dfl hs = df_add(ld(w.H[DIR][m], p), ld(w.H[DIR][m], p + sd));
    G[m] = df_sub(df_fma(b2, e3, hs), df_mul(a32, d1));
  }
}

// Blocks of 32 x 16 threads, two per SM (64 registers): 19.2 ms per launch on 1000 x 400 x 500,
// against 19.9 for 32 x 8 at five per SM (48 registers, a few spilled), 20.0 for 32 x 12 at
// three, 21.3 for 32 x 4 at ten, 22.7 for 32 x 16 at three (40 registers) and 31.9 for 32 x 8
// at three when the face fluxes of the three directions were held in registers across the
// barrier (80 registers).
template <int MODE>
__global__ void __launch_bounds__(FX* FY, 2) k_faces_update_df(Dims d, ConstsDF c, Work64 w, QDF qdf, const double* invV,
                                                            State qin, State qn, State qout, const Scalars* sc,
                                                            double alpha, int want_res, double* rhs_flat,
                                                            double* res_sum, int kchunk) {
  __shared__ float2 g1s[2][5][FY][FX];   // faces j + 1/2 of the plane, two planes in turn
  __shared__ float2 g2s[5][FY][FX];      // each thread's face k - 1/2
  const int x = threadIdx.x, y = threadIdx.y;
  const int i = (int)blockIdx.x * (FX - 1) - 1 + x, j = (int)blockIdx.y * (FY - 1) - 1 + y;
  const int k0 = (int)blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nk);
  const bool inside = i <= d.ni - 1 && j <= d.nj - 1;     // i, j >= -1 by construction
  const bool need0 = inside && y > 0;                      // face i + 1/2: halo column and body
  const bool need1 = inside && x > 0;                      // face j + 1/2: halo row and body
  const bool node = need0 && x > 0;                        // a real node this block updates
  const bool adv = advanced(d, i, j);
  const long long N = (long long)d.ni * d.nj * d.nk;
  double r2 = 0.0;
  if (node) {
    dfl g[5];
    face_df<2>(c, w, qdf, pidx(d, i, j, k0 - 1), d.sk, g);
#pragma unroll
    for (int m = 0; m < 5; ++m) g2s[m][y][x] = make_float2(g[m].hi, g[m].lo);
  }
  for (int k = k0; k < k1; ++k) {
    const long long p = pidx(d, i, j, k);
    const int b = k & 1;
    dfl g[5] = {}, a[5], cc[5];
    if (need0) face_df<0>(c, w, qdf, p, 1, g);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const float lh = __shfl_up_sync(0xffffffffu, g[m].hi, 1), ll = __shfl_up_sync(0xffffffffu, g[m].lo, 1);
      a[m] = df_sub(g[m], df_make(lh, ll));
    }
    if (need1) {
      face_df<1>(c, w, qdf, p, d.sj, g);
#pragma unroll
      for (int m = 0; m < 5; ++m) g1s[b][m][y][x] = make_float2(g[m].hi, g[m].lo);
    }
    if (node) {
      face_df<2>(c, w, qdf, p, d.sk, g);
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const float2 o = g2s[m][y][x];
        cc[m] = df_sub(g[m], df_make(o.x, o.y));
        g2s[m][y][x] = make_float2(g[m].hi, g[m].lo);
      }
    }
    __syncthreads();
    if (node) {
      double R[5];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const float2 t1 = g1s[b][m][y][x], t0 = g1s[b][m][y - 1][x];
        const dfl bb = df_sub(df_make(t1.x, t1.y), df_make(t0.x, t0.y));
        R[m] = df_to_f64(df_add(df_add(a[m], bb), cc[m]));
      }
      const double hV = 0.5 * invV[p];
      if (MODE == 0) {
        const double adtV = alpha * sc->dt * hV;
#pragma unroll
        for (int m = 0; m < 5; ++m) qout.q[m][p] = adv ? fma(-adtV, R[m], qn.q[m][p]) : qin.q[m][p];
      } else {
        const long long t = ((long long)k * d.nj + j) * d.ni + i;
#pragma unroll
        for (int m = 0; m < 5; ++m) rhs_flat[m * N + t] = adv ? R[m] * hV : 0.0;
      }
      if (adv) {
        const double r0 = R[0] * hV;
        r2 += r0 * r0;
      }
    }
  }
  if (want_res) {
    __shared__ double red[FX * FY / 32];
    const int tid = y * FX + x;
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if ((tid & 31) == 0) red[tid >> 5] = r2;
    __syncthreads();
    if (tid < 32) {
      double v = tid < FX * FY / 32 ? red[tid] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (tid == 0) atomicAdd(res_sum, v);
    }
  }
}

// FP64 metrics -> double-float copies (every padded node).
__global__ void k_metrics_df(Dims d, GridDev g, DFMetrics M) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= d.Np) return;
  for (int c = 0; c < 9; ++c) df_store(M.S[c], p, df_of(g.S[c][p]));
  for (int c = 0; c < 3; ++c) df_store(M.Smag[c], p, df_of(g.Smag[c][p]));
  df_store(M.invV, p, df_of(g.invV[p]));
  df_store(M.Delta, p, df_of(g.Delta[p]));
}


dim3 grid3(int ei, int ej, int ek) { return dim3((ei + BX - 1) / BX, (ej + BY - 1) / BY, ek); }

}  // namespace

cudaError_t metrics_to_df(const Dims& d, const GridDev& g, const DFMetrics& M, cudaStream_t st) {
  k_metrics_df<<<blocks_for(d.Np, 256), 256, 0, st>>>(d, g, M);
  return cudaGetLastError();
}

cudaError_t nodal_df(const Dims& d, const Consts& c, const DFMetrics& M, const Work64& w, const QDF& qdf,
                     const State& qin, cudaStream_t st, double* rate_max) {
  k_nodal_df<<<grid3(d.ni + 2 * kG, d.nj + 2 * kG, d.nk + 2 * kG), dim3(BX, BY), 0, st>>>(d, make_cdf(c), M, w, qin,
                                                                                          qdf, rate_max);
  return cudaGetLastError();
}

cudaError_t viscous_df(const Dims& d, const Consts& c, const DFMetrics& M, const Work64& w, const QDF& qdf,
                       cudaStream_t st) {
  k_viscous_df<<<grid3(d.ni + 2, d.nj + 2, d.nk + 2), dim3(BX, BY), 0, st>>>(d, make_cdf(c), M, w, qdf);
  return cudaGetLastError();
}

// planes per block of the faces-update kernel: enough blocks for several waves, one extra
// k-face per chunk
int faces_kchunk(const Dims& d) {
  const long long tiles = (long long)((d.ni + FX - 2) / (FX - 1)) * ((d.nj + FY - 2) / (FY - 1));
  int kc = 32;
  while (kc > 4 && tiles * ((d.nk + kc - 1) / kc) < 8 * 152) kc /= 2;
  return kc;
}

cudaError_t faces_update_df(const Dims& d, const Consts& c, const GridDev& g, const Work64& w, const QDF& qdf,
                            const State& qin, const State& qn, const State& qout, const Scalars* sc, double alpha,
                            int want_res, double* rhs_flat, cudaStream_t st) {
  double* res_sum = const_cast<double*>(&sc->res_sum);
  const int kc = faces_kchunk(d);
  const dim3 gr((d.ni + FX - 2) / (FX - 1), (d.nj + FY - 2) / (FY - 1), (d.nk + kc - 1) / kc), blk(FX, FY);
  const ConstsDF cdf = make_cdf(c);
  if (rhs_flat)
    k_faces_update_df<1><<<gr, blk, 0, st>>>(d, cdf, w, qdf, g.invV, qin, qn, qout, sc, alpha, 0, rhs_flat, res_sum, kc);
  else
    k_faces_update_df<0><<<gr, blk, 0, st>>>(d, cdf, w, qdf, g.invV, qin, qn, qout, sc, alpha, want_res, nullptr,
                                             res_sum, kc);
  return cudaGetLastError();
}

}  // namespace jz
