// Double-float constants and field access shared by the pair-form kernels (jz_stagedf.cu) and
// the pair-form transposed kernels of the adjoint (jz_adjointdf.cu).
#pragma once

#include "jz_df.cuh"
#include "jz_internal.cuh"

namespace jz {

// Constants as pairs (hi, lo) of their FP64 values: an FP32 constant such as 0.4 would put an
// error of ~1e-8 into every product.
struct ConstsDF {
  dfl gamma, gm1, gm1_half, S_hat, kappa2, kappa4, C_s, k_lam, k_sgs;
  dfl mu_sut;        // mu_ref (1 + S_hat)
  dfl third;         // 1/3
  int sigma_is_two_thirds;
  double sigma;
};

__device__ __forceinline__ dfl ld(const double* a, long long p) { return df_load(reinterpret_cast<const float2*>(a), p); }
__device__ __forceinline__ void st(double* a, long long p, dfl v) { df_store(reinterpret_cast<float2*>(a), p, v); }

// Anisotropic spectral radius lambda_d + lambda_d^(1-sigma) (lambda_e^sigma + lambda_f^sigma).
__device__ __forceinline__ void aniso_df(const ConstsDF& c, const dfl lam[3], dfl Lam[3]) {
  dfl lo[3], hi[3];
  if (c.sigma_is_two_thirds) {
    for (int d = 0; d < 3; ++d) df_cbrt_pair(lam[d], lo[d], hi[d]);
  } else {
    // a general exponent through FP64 pow (not on the benchmark path)
    for (int d = 0; d < 3; ++d) {
      const double l = df_to_f64(lam[d]);
      lo[d] = df_of(l > 0.0 ? pow(l, 1.0 - c.sigma) : 0.0);
      hi[d] = df_of(l > 0.0 ? pow(l, c.sigma) : 0.0);
    }
  }
  Lam[0] = df_fma(lo[0], df_add(hi[1], hi[2]), lam[0]);
  Lam[1] = df_fma(lo[1], df_add(hi[0], hi[2]), lam[1]);
  Lam[2] = df_fma(lo[2], df_add(hi[0], hi[1]), lam[2]);
}

// FP64 value -> pair (hi the FP32 rounding, lo the FP32 rounding of the rest), on the host.
inline dfl pair_of(double x) {
  const float h = (float)x;
  return dfl{h, (float)(x - (double)h)};
}

inline ConstsDF make_cdf(const Consts& c) {
  ConstsDF f;
  f.gamma = pair_of(c.gamma);
  f.gm1 = pair_of(c.gm1);
  f.gm1_half = pair_of(c.gm1_half);
  f.S_hat = pair_of(c.S_hat);
  f.kappa2 = pair_of(c.kappa2);
  f.kappa4 = pair_of(c.kappa4);
  f.C_s = pair_of(c.C_s);
  f.k_lam = pair_of(c.k_lam);
  f.k_sgs = pair_of(c.k_sgs);
  f.mu_sut = pair_of(c.mu_sut);
  f.third = pair_of(1.0 / 3.0);
  f.sigma_is_two_thirds = c.sigma_is_two_thirds;
  f.sigma = c.sigma;
  return f;
}

}  // namespace jz
