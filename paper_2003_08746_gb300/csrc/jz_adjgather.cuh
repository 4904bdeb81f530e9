// Gathers of the transposed nodal pass of the discrete adjoint (jz_adjoint.cu): what node
// (i, j, k) receives from the transposed viscous, sensor, inviscid-flux, spectral-radius and
// dissipation terms of its neighbours, summed in FP64.  The pair form (jz_adjointdf.cu) shares
// the padded-box test and sums the same terms in double-float on its pair arrays.
#pragma once

#include "jz_internal.cuh"

namespace jz {

__device__ __forceinline__ bool in_box(const Dims& d, int i, int j, int k) {
  return i >= -kG && i <= d.ni + 1 && j >= -kG && j <= d.nj + 1 && k >= -kG && k <= d.nk + 1;
}

// value of a padded field at (i, j, k) + offset along dir, 0 outside the padded box
__device__ __forceinline__ double nb(const Dims& d, const double* f, int i, int j, int k, int dir, int off) {
  int ii = i, jj = j, kk = k;
  if (dir == 0) ii += off; else if (dir == 1) jj += off; else kk += off;
  return in_box(d, ii, jj, kk) ? f[pidx(d, ii, jj, kk)] : 0.0;
}

struct NodalGathers {
  double fb[4];        // adjoints of u, v, w, T
  double pb;           // adjoint of p (sensors)
  double Eb[3][5];     // adjoints of the inviscid fluxes E^dir
  double Lamb[3];      // adjoints of the anisotropic spectral radii
  double qb[5];        // adjoint of Q from the dissipation and the eddy viscosity
  double mub;          // adjoint of the Sutherland viscosity
};

__device__ __forceinline__ void nodal_gathers(const Dims& d, const Adj64& a, int i, int j, int k, NodalGathers& G) {
  for (int n = 0; n < 4; ++n) {
    double v = n < 3 ? nb(d, a.ubd[n], i, j, k, 0, 0) : 0.0;
    for (int dir = 0; dir < 3; ++dir)
      v += 0.5 * (nb(d, a.G[n][dir], i, j, k, dir, -1) - nb(d, a.G[n][dir], i, j, k, dir, 1));
    G.fb[n] = v;
  }
  G.pb = 0.0;
  for (int dir = 0; dir < 3; ++dir)
    G.pb += nb(d, a.c0[dir], i, j, k, 0, 0) + nb(d, a.cpm[dir], i, j, k, dir, -1) + nb(d, a.cpm[dir], i, j, k, dir, 1);
  for (int dir = 0; dir < 3; ++dir) {
    for (int m = 0; m < 5; ++m)
      G.Eb[dir][m] = 0.5 * (nb(d, a.acc[m], i, j, k, dir, -1) - nb(d, a.acc[m], i, j, k, dir, 1));
    G.Lamb[dir] = nb(d, a.lfh[dir], i, j, k, 0, 0) + nb(d, a.lfh[dir], i, j, k, dir, -1);
  }
  // dissipation: node n receives, from faces n-2 .. n+1 (f = face n + o), the adjoints of the
  // differences it enters: d3(f-2) + d1(f-1) - 3 d3(f-1) - d1(f) + 3 d3(f) - d3(f+1), with
  // d1(f) = Db(f) ca2(f), d3(f) = -Db(f) ca4(f), Db(f) = acc(f+1) - acc(f) (zero beyond the box)
  for (int m = 0; m < 5; ++m) G.qb[m] = 0.0;
  for (int dir = 0; dir < 3; ++dir) {
    double c2[4], c4[4];           // faces n-2, n-1, n, n+1
    for (int o = 0; o < 4; ++o) {
      c2[o] = nb(d, a.ca2[dir], i, j, k, dir, o - 2);
      c4[o] = nb(d, a.ca4[dir], i, j, k, dir, o - 2);
    }
    for (int m = 0; m < 5; ++m) {
      const double am2 = nb(d, a.acc[m], i, j, k, dir, -2), am1 = nb(d, a.acc[m], i, j, k, dir, -1),
                   a0 = nb(d, a.acc[m], i, j, k, 0, 0), ap1 = nb(d, a.acc[m], i, j, k, dir, 1),
                   ap2 = nb(d, a.acc[m], i, j, k, dir, 2);
      const double D0 = am1 - am2, D1 = a0 - am1, D2 = ap1 - a0, D3 = ap2 - ap1;
      G.qb[m] += -D0 * c4[0] + D1 * c2[1] + 3.0 * (D1 * c4[1]) - D2 * c2[2] - 3.0 * (D2 * c4[2]) + D3 * c4[3];
    }
  }
  G.qb[0] += nb(d, a.rhob, i, j, k, 0, 0);
  G.mub = nb(d, a.mub, i, j, k, 0, 0);
}

}  // namespace jz
