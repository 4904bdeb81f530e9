// Grid set-up kernels: ghost coordinates, metrics of the curvilinear
// transformation (Algorithm 2: Calc(Jacob., Metric)), ghost fills and the
// copies between unpadded caller arrays and the padded device layout.
#include "jz_internal.cuh"

namespace jz {
namespace {

constexpr int kTPB = 256;

struct Ptrs16 {
  double* p[16];
};

__device__ __forceinline__ long long ridx(const Dims& d, int i, int j, int k) {
  return ((long long)k * d.nj + j) * d.ni + i;   // unpadded real index
}

__device__ __forceinline__ int wrapk(const Dims& d, int k) { return ((k % d.nk) + d.nk) % d.nk; }

// Jet coordinates for a real axial index ir: azimuthal wrap, across-axis
// mirror (node (ir, -j, k + nk/2)), linear extrapolation beyond the far field.
__device__ double jet_base(const Dims& d, const double* x, int ir, int j, int k) {
  if (j < 0) return x[ridx(d, ir, -j, wrapk(d, k + d.nk / 2))];
  if (j >= d.nj) {
    const int m = j - (d.nj - 1);
    const double a = x[ridx(d, ir, d.nj - 1, wrapk(d, k))];
    const double b = x[ridx(d, ir, d.nj - 2, wrapk(d, k))];
    return (1 + m) * a - m * b;
  }
  return x[ridx(d, ir, j, wrapk(d, k))];
}

__global__ void k_pad_coords(Dims d, const double* __restrict__ xr, double px0, double px1, double px2,
                             double py0, double py1, double py2, double pz0, double pz1, double pz2,
                             Ptrs16 out) {
  Box b{-kG, -kG, -kG, d.ni + 2 * kG, d.nj + 2 * kG, d.nk + 2 * kG};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const long long N = (long long)d.ni * d.nj * d.nk;
  const double per[3][3] = {{px0, px1, px2}, {py0, py1, py2}, {pz0, pz1, pz2}};
  for (int c = 0; c < 3; ++c) {
    const double* x = xr + c * N;
    double v;
    if (d.topo == JZ_TOPO_PERIODIC) {
      int si, sj, sk;
      ghost_source(d, i, j, k, si, sj, sk);
      const double wi = (double)((i - si) / d.ni), wj = (double)((j - sj) / d.nj),
                   wk = (double)((k - sk) / d.nk);
      v = x[ridx(d, si, sj, sk)];
      v = v + wi * per[0][c];
      v = v + wj * per[1][c];
      v = v + wk * per[2][c];
    } else {
      if (i < 0) {
        const int m = -i;
        v = (1 + m) * jet_base(d, x, 0, j, k) - m * jet_base(d, x, 1, j, k);
      } else if (i >= d.ni) {
        const int m = i - (d.ni - 1);
        v = (1 + m) * jet_base(d, x, d.ni - 1, j, k) - m * jet_base(d, x, d.ni - 2, j, k);
      } else {
        v = jet_base(d, x, i, j, k);
      }
    }
    out.p[c][p] = v;
  }
}

// C_dir = r_dir x r on the nodes within one layer of the real region.
__global__ void k_cross(Dims d, Ptrs16 X, Ptrs16 C) {
  Box b{-1, -1, -1, d.ni + 2, d.nj + 2, d.nk + 2};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const long long s[3] = {1, d.sj, d.sk};
  const double r[3] = {X.p[0][p], X.p[1][p], X.p[2][p]};
  for (int dir = 0; dir < 3; ++dir) {
    double a[3];
    for (int c = 0; c < 3; ++c) a[c] = 0.5 * (X.p[c][p + s[dir]] - X.p[c][p - s[dir]]);
    C.p[3 * dir + 0][p] = a[1] * r[2] - a[2] * r[1];
    C.p[3 * dir + 1][p] = a[2] * r[0] - a[0] * r[2];
    C.p[3 * dir + 2][p] = a[0] * r[1] - a[1] * r[0];
  }
}

// Symmetric conservative metrics and the volume on the real nodes:
//   S^xi = [d_zeta(C_eta) - d_eta(C_zeta)]/2, S^eta = [d_xi(C_zeta) - d_zeta(C_xi)]/2,
//   S^zeta = [d_eta(C_xi) - d_xi(C_eta)]/2, V = r_xi . (r_eta x r_zeta).
__global__ void k_metrics(Dims d, Ptrs16 X, Ptrs16 C, Ptrs16 M) {
  Box b{0, 0, 0, d.ni, d.nj, d.nk};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  const long long s[3] = {1, d.sj, d.sk};
  auto dd = [&](const double* f, int dir) { return 0.5 * (f[p + s[dir]] - f[p - s[dir]]); };
  // (dir, first, second): S^dir = 0.5 * (d_first(C_a) - d_second(C_b))
  const int first[3] = {2, 0, 1};   // zeta, xi, eta
  const int ca[3] = {1, 2, 0};      // C_eta, C_zeta, C_xi
  const int second[3] = {1, 2, 0};  // eta, zeta, xi
  const int cb[3] = {2, 0, 1};      // C_zeta, C_xi, C_eta
  for (int dir = 0; dir < 3; ++dir)
    for (int c = 0; c < 3; ++c)
      M.p[3 * dir + c][p] = 0.5 * (dd(C.p[3 * ca[dir] + c], first[dir]) - dd(C.p[3 * cb[dir] + c], second[dir]));
  double a[3][3];
  for (int dir = 0; dir < 3; ++dir)
    for (int c = 0; c < 3; ++c) a[dir][c] = dd(X.p[c], dir);
  const double cx = a[1][1] * a[2][2] - a[1][2] * a[2][1];
  const double cy = a[1][2] * a[2][0] - a[1][0] * a[2][2];
  const double cz = a[1][0] * a[2][1] - a[1][1] * a[2][0];
  double V = a[0][0] * cx;
  V = V + a[0][1] * cy;
  V = V + a[0][2] * cz;
  M.p[9][p] = V;
}

__global__ void k_derived(Dims d, Ptrs16 M, Ptrs16 out) {
  Box b{-kG, -kG, -kG, d.ni + 2 * kG, d.nj + 2 * kG, d.nk + 2 * kG};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long p = pidx(d, i, j, k);
  for (int dir = 0; dir < 3; ++dir) {
    const double x = M.p[3 * dir][p], y = M.p[3 * dir + 1][p], z = M.p[3 * dir + 2][p];
    out.p[dir][p] = sqrt(x * x + y * y + z * z);
  }
  const double V = M.p[9][p];
  out.p[3][p] = V > 0.0 ? 1.0 / V : 0.0;
  out.p[4][p] = cbrt(V);
}

// Ghost shell enumerated directly: the four k-ghost planes (with their i/j
// ghosts), then the four j-ghost rows of every real k, then the four i-ghost
// columns of every real (j, k).  Every ghost copies from a real node.
__device__ __forceinline__ bool ghost_coord(const Dims& d, long long t, int& i, int& j, int& k) {
  const long long ei = d.ni + 2 * kG, ej = d.nj + 2 * kG;
  const long long nA = 4 * ei * ej, nB = 4 * ei * d.nk, nC = 4LL * d.nj * d.nk;
  if (t < nA) {
    i = (int)(t % ei) - kG;
    const long long r = t / ei;
    j = (int)(r % ej) - kG;
    const int s = (int)(r / ej);                 // 0..3
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

__global__ void k_ghost_fill(Dims d, Ptrs16 f, int nvar) {
  int i, j, k;
  if (!ghost_coord(d, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  int si, sj, sk;
  ghost_source(d, i, j, k, si, sj, sk);
  const long long p = pidx(d, i, j, k), q = pidx(d, si, sj, sk);
  for (int v = 0; v < nvar; ++v) f.p[v][p] = f.p[v][q];
}

// FP32 metric records: kMF floats per padded node from kMF FP64 arrays.
__global__ void k_to_f32(Dims d, Ptrs16 src, float* __restrict__ dst) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= d.Np) return;
  float r[kMF];
  for (int v = 0; v < kMF; ++v) r[v] = __double2float_rn(src.p[v][t]);
  float4* o = reinterpret_cast<float4*>(dst + t * kMF);
  o[0] = make_float4(r[0], r[1], r[2], r[3]);
  o[1] = make_float4(r[4], r[5], r[6], r[7]);
  o[2] = make_float4(r[8], r[9], r[10], r[11]);
}

__global__ void k_pack(Dims d, Ptrs16 padded, const double* __restrict__ flat, int nvar) {
  Box b{0, 0, 0, d.ni, d.nj, d.nk};
  int i, j, k;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (!box_coord(b, t, i, j, k)) return;
  const long long N = (long long)d.ni * d.nj * d.nk, p = pidx(d, i, j, k);
  for (int v = 0; v < nvar; ++v) padded.p[v][p] = flat[v * N + t];
}

__global__ void k_unpack(Dims d, Ptrs16 padded, double* __restrict__ flat, int nvar) {
  Box b{0, 0, 0, d.ni, d.nj, d.nk};
  int i, j, k;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (!box_coord(b, t, i, j, k)) return;
  const long long N = (long long)d.ni * d.nj * d.nk, p = pidx(d, i, j, k);
  for (int v = 0; v < nvar; ++v) flat[v * N + t] = padded.p[v][p];
}

__global__ void k_check_volume(Dims d, Ptrs16 M, int* bad) {
  Box b{0, 0, 0, d.ni, d.nj, d.nk};
  int i, j, k;
  if (!box_coord(b, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  if (d.topo == JZ_TOPO_JET && (i == 0 || i == d.ni - 1 || j == 0 || j == d.nj - 1)) return;
  const double V = M.p[9][pidx(d, i, j, k)];
  if (!(V > 0.0)) atomicAdd(bad, 1);
}

Ptrs16 ptrs(double* const* a, int n) {
  Ptrs16 p{};
  for (int i = 0; i < n; ++i) p.p[i] = a[i];
  return p;
}

}  // namespace

cudaError_t pad_coordinates(const Dims& d, const double* xyz_real, const double* period, GridDev& g,
                            cudaStream_t st) {
  double per[9] = {0};
  if (period)
    for (int i = 0; i < 9; ++i) per[i] = period[i];
  const long long n = (long long)(d.ni + 2 * kG) * (d.nj + 2 * kG) * (d.nk + 2 * kG);
  k_pad_coords<<<blocks_for(n, kTPB), kTPB, 0, st>>>(d, xyz_real, per[0], per[1], per[2], per[3], per[4],
                                                      per[5], per[6], per[7], per[8], ptrs(g.xyz, 3));
  return cudaGetLastError();
}

cudaError_t compute_metrics(const Dims& d, GridDev& g, double* scratch9[9], cudaStream_t st) {
  const long long n1 = (long long)(d.ni + 2) * (d.nj + 2) * (d.nk + 2);
  k_cross<<<blocks_for(n1, kTPB), kTPB, 0, st>>>(d, ptrs(g.xyz, 3), ptrs(scratch9, 9));
  double* M[10];
  for (int i = 0; i < 9; ++i) M[i] = g.S[i];
  M[9] = g.V;
  const long long nr = (long long)d.ni * d.nj * d.nk;
  k_metrics<<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, ptrs(g.xyz, 3), ptrs(scratch9, 9), ptrs(M, 10));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = ghost_fill(d, M, 10, st);
  if (e != cudaSuccess) return e;
  double* out[5] = {g.Smag[0], g.Smag[1], g.Smag[2], g.invV, g.Delta};
  const long long np = (long long)(d.ni + 2 * kG) * (d.nj + 2 * kG) * (d.nk + 2 * kG);
  k_derived<<<blocks_for(np, kTPB), kTPB, 0, st>>>(d, ptrs(M, 10), ptrs(out, 5));
  return cudaGetLastError();
}

cudaError_t check_volume(const Dims& d, const GridDev& g, int* bad, cudaStream_t st) {
  double* M[10];
  for (int i = 0; i < 9; ++i) M[i] = g.S[i];
  M[9] = g.V;
  const long long nr = (long long)d.ni * d.nj * d.nk;
  k_check_volume<<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, ptrs(M, 10), bad);
  return cudaGetLastError();
}

cudaError_t ghost_fill(const Dims& d, double* const* f, int nvar, cudaStream_t st) {
  const long long ei = d.ni + 2 * kG, ej = d.nj + 2 * kG;
  const long long ng = 4 * ei * ej + 4 * ei * d.nk + 4LL * d.nj * d.nk;
  k_ghost_fill<<<blocks_for(ng, kTPB), kTPB, 0, st>>>(d, ptrs(f, nvar), nvar);
  return cudaGetLastError();
}

// Surface copies: the far-field normals S^eta at j = nj-1 ([3][nk][ni]) and the
// entrance-plane coordinates y, z at i = 0 ([2][nk][nj]).
__global__ void k_boundary_copies(Dims d, GridDev g) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nb = (long long)d.nk * d.ni, ne = (long long)d.nk * d.nj;
  if (t < 3 * nb) {
    const int c = (int)(t / nb);
    const long long r = t % nb;
    const int k = (int)(r / d.ni), i = (int)(r % d.ni);
    g.Sb[t] = g.S[3 + c][pidx(d, i, d.nj - 1, k)];
  } else if (t < 3 * nb + 2 * ne) {
    const long long u = t - 3 * nb;
    const int c = (int)(u / ne);
    const long long r = u % ne;
    const int k = (int)(r / d.nj), j = (int)(r % d.nj);
    g.Xin[u] = g.xyz[1 + c][pidx(d, 0, j, k)];
  }
}

cudaError_t boundary_copies(const Dims& d, const GridDev& g, cudaStream_t st) {
  const long long n = 3LL * d.nk * d.ni + 2LL * d.nk * d.nj;
  k_boundary_copies<<<blocks_for(n, kTPB), kTPB, 0, st>>>(d, g);
  return cudaGetLastError();
}

cudaError_t metrics_to_f32(const Dims& d, const GridDev& g, float* Mf, cudaStream_t st) {
  double* M[kMF];
  for (int i = 0; i < 9; ++i) M[i] = g.S[i];
  M[MF_V] = g.V;
  M[MF_IV] = g.invV;
  M[MF_D] = g.Delta;
  k_to_f32<<<blocks_for(d.Np, kTPB), kTPB, 0, st>>>(d, ptrs(M, kMF), Mf);
  return cudaGetLastError();
}

cudaError_t pack_real(const Dims& d, double* const* padded, const double* flat, int nvar, cudaStream_t st) {
  const long long nr = (long long)d.ni * d.nj * d.nk;
  k_pack<<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, ptrs(padded, nvar), flat, nvar);
  return cudaGetLastError();
}

cudaError_t unpack_real(const Dims& d, double* const* padded, double* flat, int nvar, cudaStream_t st) {
  const long long nr = (long long)d.ni * d.nj * d.nk;
  k_unpack<<<blocks_for(nr, kTPB), kTPB, 0, st>>>(d, ptrs(padded, nvar), flat, nvar);
  return cudaGetLastError();
}

}  // namespace jz
