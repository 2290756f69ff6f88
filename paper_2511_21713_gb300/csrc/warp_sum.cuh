// Fixed-order sum of a strided run of float64 values by one warp.
#pragma once

namespace pbfb {
namespace {

// p[0] + p[s] + ... + p[(n-1) s]: lane l adds entries l, l + 32, ... in that order, eight loads in
// flight at a time, then a xor butterfly over the 32 lanes (every lane returns the same value).
// Call with all 32 lanes of the warp.
__device__ __forceinline__ double warp_strided_sum(const double* __restrict__ p, int n, long long s) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int k0 = lane; k0 < n; k0 += 32 * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + 32 * u;
      v[u] = k < n ? p[k * s] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + 32 * u < n) acc += v[u];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

}  // namespace
}  // namespace pbfb
