// Shared-memory Stockham FFT on batches of lines (device code).
//
// Decimation-in-frequency Stockham autosort: at a stage with radix r, current
// sub-length n = len / s (s = product of the radices already applied) and
// m = n / r, butterfly (p, q) with p < m, q < s reads x[q + s (p + t m)],
// t < r, forms the r-point DFT and writes
//   y[q + s (r p + u)] = DFT_r(a)[u] * w_n^(p u),   w_n = exp(-2 pi i / n),
// and w_n^(p u) = w_len^(p u s) is read from a table of len twiddles.  Input
// and output are in natural order; the buffers alternate between stages.
#pragma once

#include "vie_internal.cuh"

namespace vie {

// DFT_r constants (exact values of cos/sin at rational multiples of pi).
template <typename R> struct RadixConst;
template <> struct RadixConst<float> {
  static constexpr float s3 = 0.86602540378443864676f;       // sqrt(3)/2
  static constexpr float c51 = 0.30901699437494742410f;      // (sqrt5 - 1)/4
  static constexpr float c52 = -0.80901699437494742410f;     // -(sqrt5 + 1)/4
  static constexpr float s51 = 0.95105651629515357212f;      // sqrt((5 + sqrt5)/8)
  static constexpr float s52 = 0.58778525229247312917f;      // sqrt((5 - sqrt5)/8)
};
template <> struct RadixConst<double> {
  static constexpr double s3 = 0.86602540378443864676;
  static constexpr double c51 = 0.30901699437494742410;
  static constexpr double c52 = -0.80901699437494742410;
  static constexpr double s51 = 0.95105651629515357212;
  static constexpr double s52 = 0.58778525229247312917;
};

template <typename V> struct real_of;
template <> struct real_of<float2> { typedef float type; };
template <> struct real_of<double2> { typedef double type; };

// In-place r-point DFT of a[0..r); INV selects exp(+2 pi i tu / r).
template <typename V, bool INV>
__device__ __forceinline__ void dft_small(V* a, int r) {
  typedef typename real_of<V>::type R;
  switch (r) {
    case 2: {
      V b0 = add(a[0], a[1]), b1 = sub(a[0], a[1]);
      a[0] = b0; a[1] = b1;
      break;
    }
    case 3: {
      V s = add(a[1], a[2]), d = sub(a[1], a[2]);
      V m = sub(a[0], scale(s, R(0.5)));
      V t = scale(d, RadixConst<R>::s3);
      V it = INV ? mul_pi(t) : mul_mi(t);   // -/+ i s3 (a1 - a2)
      a[0] = add(a[0], s);
      a[1] = add(m, it);
      a[2] = sub(m, it);
      break;
    }
    case 4: {
      V s02 = add(a[0], a[2]), d02 = sub(a[0], a[2]);
      V s13 = add(a[1], a[3]), d13 = sub(a[1], a[3]);
      V id = INV ? mul_pi(d13) : mul_mi(d13);
      a[0] = add(s02, s13);
      a[2] = sub(s02, s13);
      a[1] = add(d02, id);
      a[3] = sub(d02, id);
      break;
    }
    case 5: {
      const R c1 = RadixConst<R>::c51, c2 = RadixConst<R>::c52;
      const R s1 = RadixConst<R>::s51, s2 = RadixConst<R>::s52;
      V s14 = add(a[1], a[4]), d14 = sub(a[1], a[4]);
      V s23 = add(a[2], a[3]), d23 = sub(a[2], a[3]);
      V m1 = add(a[0], add(scale(s14, c1), scale(s23, c2)));
      V m2 = add(a[0], add(scale(s14, c2), scale(s23, c1)));
      V t1 = add(scale(d14, s1), scale(d23, s2));
      V t2 = sub(scale(d14, s2), scale(d23, s1));
      V i1 = INV ? mul_pi(t1) : mul_mi(t1);
      V i2 = INV ? mul_pi(t2) : mul_mi(t2);
      a[0] = add(a[0], add(s14, s23));
      a[1] = add(m1, i1);
      a[4] = sub(m1, i1);
      a[2] = add(m2, i2);
      a[3] = sub(m2, i2);
      break;
    }
    default:
      break;
  }
}

// One Stockham stage of a radix r above 5 (any r that divides len): the
// r-point DFT of each butterfly is summed directly, its roots of unity
// exp(-2 pi i t u / r) = tw[((t u) mod r) (len / r)] read from the length-len
// table, O(r^2) per butterfly.  Lets lengths with prime factors such as 7,
// 11 or 13 use the same kernels as 5-smooth lengths.
template <typename V, bool INV>
__device__ __forceinline__ void stockham_stage_generic(const V* __restrict__ src, V* __restrict__ dst,
                                                       int len, int pitch, int nlines, int r, int s,
                                                       const V* __restrict__ tw, int tid, int nth) {
  const int n = len / s;
  const int m = n / r;
  const int nb = len / r;
  const int step = len / r;
  const int total = nb * nlines;
  for (int idx = tid; idx < total; idx += nth) {
    const int line = idx / nb;
    const int b = idx - line * nb;
    const int p = b / s;
    const int q = b - p * s;
    const V* x = src + line * pitch;
    V* y = dst + line * pitch;
    for (int u = 0; u < r; ++u) {
      V acc = x[q + s * p];
      int e = 0;                       // (t u) mod r, advanced by u per term
      for (int t = 1; t < r; ++t) {
        e += u;
        if (e >= r) e -= r;
        const V w = tw[e * step];
        const V a = x[q + s * (p + t * m)];
        acc = add(acc, INV ? mulc(a, w) : mul(a, w));
      }
      if (u > 0) {
        const V w = tw[p * u * s];
        acc = INV ? mulc(acc, w) : mul(acc, w);
      }
      y[q + s * (r * p + u)] = acc;
    }
  }
}

// One Stockham stage over `nlines` lines (line pitch `pitch`); radices above
// 5 only when GENERIC (the operator's passes use 5-smooth lengths).
template <typename V, bool INV, bool GENERIC = false>
__device__ __forceinline__ void stockham_stage(const V* __restrict__ src, V* __restrict__ dst,
                                               int len, int pitch, int nlines, int r, int s,
                                               const V* __restrict__ tw, int tid, int nth) {
  if (GENERIC && r > 5) {
    stockham_stage_generic<V, INV>(src, dst, len, pitch, nlines, r, s, tw, tid, nth);
    return;
  }
  const int n = len / s;
  const int m = n / r;
  const int nb = len / r;
  const int total = nb * nlines;
  for (int idx = tid; idx < total; idx += nth) {
    const int line = idx / nb;
    const int b = idx - line * nb;
    const int p = b / s;
    const int q = b - p * s;
    const V* x = src + line * pitch;
    V* y = dst + line * pitch;
    V a[5];
#pragma unroll
    for (int t = 0; t < 5; ++t)
      if (t < r) a[t] = x[q + s * (p + t * m)];
    dft_small<V, INV>(a, r);
    y[q + s * (r * p)] = a[0];
#pragma unroll
    for (int u = 1; u < 5; ++u) {
      if (u < r) {
        const V w = tw[p * u * s];
        y[q + s * (r * p + u)] = INV ? mulc(a[u], w) : mul(a[u], w);
      }
    }
  }
}

// Full transform of `nlines` lines held in buf0; buf1 is scratch of the same
// shape.  Every thread of the block must call it.  Returns the buffer holding
// the result.
template <typename V, bool INV, bool GENERIC = false>
__device__ V* fft_lines(V* buf0, V* buf1, const Radices& rd, int pitch, int nlines,
                        const V* tw, int tid, int nth) {
  V* src = buf0;
  V* dst = buf1;
  int s = 1;
  for (int st = 0; st < rd.nstages; ++st) {
    const int r = rd.r[st];
    stockham_stage<V, INV, GENERIC>(src, dst, rd.len, pitch, nlines, r, s, tw, tid, nth);
    __syncthreads();
    V* t = src; src = dst; dst = t;
    s *= r;
  }
  return src;
}

}  // namespace vie
