// Self-check of the FP64 reciprocal, square root and cube roots used by the
// FP64 form (rcp64, sqrt64, cbrt_pair64) against IEEE division, IEEE sqrt and
// the CUDA math library's cbrt.
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

}  // namespace

cudaError_t math_check(double* dev_maxrel3, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(dev_maxrel3, 0, 3 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_math_check<<<kBlocks, kTPB, 0, st>>>(dev_maxrel3);
  return cudaGetLastError();
}

}  // namespace jz
