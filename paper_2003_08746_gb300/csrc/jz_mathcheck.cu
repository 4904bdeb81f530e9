// Self-check of the FP64 reciprocal, square root and cube roots used by the
// FP64 form (rcp64, sqrt64, cbrt_pair64) against IEEE division, IEEE sqrt and
// the CUDA math library's cbrt; and of the pair form's double-float
// operations (jz_df.cuh) against FP64.
#include "jz_df.cuh"
#include "jz_internal.cuh"

namespace jz {
namespace {

constexpr int kTPB = 256;
constexpr int kBlocks = 4096;     // 2^20 samples

// Sample s in [0, 2^20): x = 2^e (1 + f) with e in [-99, 99] and f in [0, 1),
// spread so that every binade of [1e-30, 1e30] gets ~5,000 mantissas.
__global__ void k_math_check(double* maxrel) {
  const unsigned s = blockIdx.x * kTPB + threadIdx.x;
  const int e = (int)(s % 199u) - 99;
  const double f = (double)((s / 199u) * 2654435761u % 1000003u) / 1000003.0;
  const double x = ldexp(1.0 + f, e);
  const double r_ref = 1.0 / x, c_ref = cbrt(x), s_ref = sqrt(x);
  double e1 = fabs(rcp64(x) - r_ref) / r_ref;
  double c1, c2;
  cbrt_pair64(x, c1, c2);
  const double c2_ref = cbrt(x * x);
  double e2 = fmax(fabs(c1 - c_ref) / c_ref, fabs(c2 - c2_ref) / c2_ref);
  double e3 = fabs(sqrt64(x) - s_ref) / s_ref;
  if (s == 0) {                                             // 0 -> 0
    cbrt_pair64(0.0, c1, c2);
    e2 = fmax(e2, fabs(c1) + fabs(c2));
    e3 = fmax(e3, fabs(sqrt64(0.0)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    e1 = fmax(e1, __shfl_xor_sync(0xffffffffu, e1, o));
    e2 = fmax(e2, __shfl_xor_sync(0xffffffffu, e2, o));
    e3 = fmax(e3, __shfl_xor_sync(0xffffffffu, e3, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(reinterpret_cast<unsigned long long*>(&maxrel[0]), (unsigned long long)__double_as_longlong(e1));
    atomicMax(reinterpret_cast<unsigned long long*>(&maxrel[1]), (unsigned long long)__double_as_longlong(e2));
    atomicMax(reinterpret_cast<unsigned long long*>(&maxrel[2]), (unsigned long long)__double_as_longlong(e3));
  }
}

// Double-float operations against FP64 on pairs of operands x, y = +-2^e (1 + f), e in [-40, 40]
// (the range the stage quantities take), plus |x| down to 1e-32 for the roots.  Errors are
// relative to the FP64 result, except for sums and differences, whose error is bounded
// relative to |x| + |y| (the cancellation of the operands is exact in neither form's inputs).
// out: [add, mul, fma, rcp, sqrt, cbrt pair, conversion round trip, sqrt and cbrt pair of
// arguments below 1e-30 (the FP32 fallbacks)]
__global__ void k_df_check(double* out) {
  const unsigned s = blockIdx.x * kTPB + threadIdx.x;
  const double f1 = (double)((s * 2654435761u) % 1000003u) / 1000003.0;
  const double f2 = (double)((s * 40503u + 17u) % 999983u) / 999983.0;
  const double f3 = (double)((s * 69069u + 5u) % 999979u) / 999979.0;
  const int e1 = (int)(s % 81u) - 40, e2 = (int)((s / 81u) % 81u) - 40, e3 = (int)((s / 6561u) % 81u) - 40;
  const double x = ((s & 1u) ? -1.0 : 1.0) * ldexp(1.0 + f1, e1);
  const double y = ((s & 2u) ? -1.0 : 1.0) * ldexp(1.0 + f2, e2);
  const double z = ((s & 4u) ? -1.0 : 1.0) * ldexp(1.0 + f3, e3);
  const dfl X = df_of(x), Y = df_of(y), Z = df_of(z);
  double err[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  err[0] = fabs(df_to_f64(df_add(X, Y)) - (x + y)) / (fabs(x) + fabs(y));
  err[1] = fabs(df_to_f64(df_mul(X, Y)) - x * y) / fabs(x * y);
  err[2] = fabs(df_to_f64(df_fma(X, Y, Z)) - fma(x, y, z)) / (fabs(x * y) + fabs(z));
  err[3] = fabs(df_to_f64(df_rcp(X)) - 1.0 / x) * fabs(x);
  const bool tiny = s % 7u == 0;
  const double ax = fabs(x) * (tiny ? ldexp(1.0, -66) : 1.0);     // 1/7 of them below 1e-30
  const dfl AX = df_of(ax);
  const double es = fabs(df_to_f64(df_sqrt(AX)) - sqrt(ax)) / sqrt(ax);
  dfl c1, c2;
  df_cbrt_pair(AX, c1, c2);
  const double ec = fmax(fabs(df_to_f64(c1) - cbrt(ax)) / cbrt(ax), fabs(df_to_f64(c2) - cbrt(ax * ax)) / cbrt(ax * ax));
  err[tiny ? 7 : 4] = es;
  err[tiny ? 8 : 5] = ec;
  err[6] = fabs(df_to_f64(X) - x) / fabs(x);
  for (int k = 0; k < 9; ++k) {
    double v = err[k];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0)
      atomicMax(reinterpret_cast<unsigned long long*>(&out[k]), (unsigned long long)__double_as_longlong(v));
  }
}

}  // namespace

cudaError_t df_check(double* dev_maxrel9, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(dev_maxrel9, 0, 9 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_df_check<<<kBlocks, kTPB, 0, st>>>(dev_maxrel9);
  return cudaGetLastError();
}

cudaError_t math_check(double* dev_maxrel3, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(dev_maxrel3, 0, 3 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_math_check<<<kBlocks, kTPB, 0, st>>>(dev_maxrel3);
  return cudaGetLastError();
}

}  // namespace jz
