// Register-resident FFT of a compile-time length L (one line per thread).
//
// Same decimation-in-frequency Stockham scheme as fft.cuh, but every index is
// a compile-time constant: the L values live in registers, each stage is a
// fixed permutation with butterflies of radix 4, 2, 3 or 5 (greedy, in that
// order), and the only memory traffic is the twiddle table
// tw[k] = exp(-2 pi i k / L) read at constant offsets.  No barriers, no
// integer division.
#pragma once

#include "fft.cuh"

namespace vie {

__host__ __device__ constexpr int first_radix(int n) {
  return (n % 4 == 0) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : 0;
}

__host__ __device__ constexpr bool reg_fft_supported(int n) {
  return n == 1 ? true : (first_radix(n) == 0 ? false : reg_fft_supported(n / first_radix(n)));
}

template <typename V, bool INV, int L, int N, int S>
struct RegStage {
  // N: current sub-length, S: product of the radices already applied
  static __device__ __forceinline__ void run(V (&a)[L], const V* __restrict__ tw) {
    constexpr int R = first_radix(N);
    static_assert(R != 0, "length must be 2^a 3^b 5^c");
    constexpr int M = N / R;
    V b[L];
#pragma unroll
    for (int p = 0; p < M; ++p) {
#pragma unroll
      for (int q = 0; q < S; ++q) {
        V t[R];
#pragma unroll
        for (int u = 0; u < R; ++u) t[u] = a[q + S * (p + u * M)];
        dft_small<V, INV>(t, R);
        b[q + S * (R * p)] = t[0];
#pragma unroll
        for (int u = 1; u < R; ++u) {
          if (p == 0) {
            b[q + S * (R * p + u)] = t[u];
          } else {
            const V w = tw[p * u * S];
            b[q + S * (R * p + u)] = INV ? mulc(t[u], w) : mul(t[u], w);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < L; ++i) a[i] = b[i];
    RegStage<V, INV, L, M, S * R>::run(a, tw);
  }
};

template <typename V, bool INV, int L, int S>
struct RegStage<V, INV, L, 1, S> {
  static __device__ __forceinline__ void run(V (&)[L], const V* __restrict__) {}
};

// In-place transform of a[0..L): forward (exp(-i)) or inverse (exp(+i), no scaling).
template <typename V, bool INV, int L>
__device__ __forceinline__ void reg_fft(V (&a)[L], const V* __restrict__ tw) {
  RegStage<V, INV, L, L, 1>::run(a, tw);
}

}  // namespace vie
