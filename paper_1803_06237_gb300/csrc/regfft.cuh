// Register-resident FFT of a compile-time length L (one line per thread).
//
// Same decimation-in-frequency Stockham scheme as fft.cuh, but every index is
// a compile-time constant: the L values live in registers, each stage is a
// fixed permutation with butterflies of radix 4, 2, 3 or 5 (greedy, in that
// order), and the twiddles exp(-2 pi i k / L) are compile-time constants (the
// table argument, tw[k] = exp(-2 pi i k / L), is no longer read).  No memory
// traffic, no barriers, no integer division.
#pragma once

#include <type_traits>

#include "fft.cuh"

namespace vie {

__host__ __device__ constexpr int first_radix(int n) {
  return (n % 4 == 0) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : 0;
}

__host__ __device__ constexpr bool reg_fft_supported(int n) {
  return n == 1 ? true : (first_radix(n) == 0 ? false : reg_fft_supported(n / first_radix(n)));
}

// exp(-2 pi i k / L) at compile time: the angle reduced to [-pi, pi], then
// the Taylor series of cos and sin (30 terms: below 1e-16 for |x| <= pi).
// The stages multiply by these constants, so no twiddle is loaded and
// multiplications by 1, -i or (1 - i)/sqrt 2 fold.
__host__ __device__ constexpr double tw_taylor(double x, bool want_sin) {
  double term = want_sin ? x : 1.0, sum = term;
  for (int n = want_sin ? 1 : 0; n < 60; n += 2) {
    term *= -x * x / ((double)(n + 1) * (double)(n + 2));
    sum += term;
  }
  return sum;
}
template <int L, int K>
struct TwConst {
  static constexpr int k = ((K % L) + L) % L;
  static constexpr int kr = 2 * k > L ? k - L : k;    // angle in [-pi, pi]
  static constexpr double x = -6.283185307179586476925286766559 * (double)kr / (double)L;
  static constexpr double c = tw_taylor(x, false);
  static constexpr double s = tw_taylor(x, true);
};
template <typename V> struct TwMake;
template <> struct TwMake<float2> {
  static __device__ __forceinline__ float2 make(double c, double s) { return make_float2((float)c, (float)s); }
};
template <> struct TwMake<double2> {
  static __device__ __forceinline__ double2 make(double c, double s) { return make_double2(c, s); }
};

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

template <typename V, bool INV, int L, int N, int S>
struct RegStage {
  // N: current sub-length, S: product of the radices already applied
  static __device__ __forceinline__ void run(V (&a)[L], const V* __restrict__ tw) {
    constexpr int R = first_radix(N);
    static_assert(R != 0, "length must be 2^a 3^b 5^c");
    constexpr int M = N / R;
    V b[L];
    static_for<0, M>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
#pragma unroll
      for (int q = 0; q < S; ++q) {
        V t[R];
#pragma unroll
        for (int u = 0; u < R; ++u) t[u] = a[q + S * (p + u * M)];
        dft_small<V, INV>(t, R);
        b[q + S * (R * p)] = t[0];
        static_for<1, R>([&](auto uc) {
          constexpr int u = decltype(uc)::value;
          if constexpr (p == 0) {
            b[q + S * (R * p + u)] = t[u];
          } else {
            // w_L^(p u S), a compile-time constant
            typedef TwConst<L, p * u * S> W;
            const V w = TwMake<V>::make(W::c, W::s);
            b[q + S * (R * p + u)] = INV ? mulc(t[u], w) : mul(t[u], w);
          }
        });
      }
    });
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
