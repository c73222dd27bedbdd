// Krylov solvers for the discrete J-VIE (I - M_eps N) w = b (Sec. 5.4 of
// arXiv:1803.06237; the paper solves it with GMRES at tolerance 1e-8, Sec. 5),
// for one problem or a batch of problems of uneven sizes.
//
// * Arnoldi with classical Gram-Schmidt and a second pass when the first
//   one lost too much of the vector (the Daniel-Gragg-Kaufman-Stewart
//   criterion ||w'|| < ||w|| / sqrt 2, decided on the device; the second pass
//   then runs as in CGS2, otherwise its kernels return at once).  Products and each thread's short partial sums use
//   the vectors' precision (FP32 for complex64: this GPU's FP64 rate is a
//   small fraction of its FP32 rate); every sum across threads and blocks is
//   FP64, in a fixed order.  The Hessenberg matrix, Givens rotations and the
//   small least-squares problem are FP64 and stay on the device.  The host
//   reads one status record per problem every few steps.
// * Right-preconditioned flexible GMRES keeps z_j = P(v_j) (a nonlinear P is
//   allowed); with no preconditioner z_j = v_j and Z aliases V.
// * Mixed precision: iterative refinement whose residual r = b - A x uses the
//   complex128 operator and whose correction solves A d = r with the
//   complex64 operator to a loose tolerance; x accumulates in complex128.
//   Plain mode runs restarted GMRES on the complex128 operator.
// * Batching: every kernel takes a table of per-problem records and
//   blockIdx.y (or blockIdx.x for per-problem kernels) selects the problem,
//   so one launch advances all open problems; the operator is applied per
//   group of equal shape (matvec_group).  Problems stop individually when
//   their true FP64 residual reaches the tolerance.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

constexpr int kDotBlocks = 456;     // 3 x 152 SMs per problem
constexpr int kThreads = 256;
constexpr int kMaxRestart = 1000;
constexpr int kMaxInnerCycles = 64;   // complex64 cycles per refinement step

struct SolveStatus {
  int active;        // 1 while the cycle should continue
  int j;             // Arnoldi steps completed in this cycle
  int converged;     // residual estimate reached the target
  int breakdown;     // h_{j+1,j} == 0 (exact solution in the subspace) or non-finite
  double beta;       // ||r|| at the start of the cycle (true residual)
  double target;     // absolute residual target of the cycle
  double resid;      // |g_{j+1}| (current residual estimate)
  double inv_h;      // 1 / h_{j+1,j}
  int reorth;        // 1: the current step needs the second Gram-Schmidt pass
  int reorth_count;  // steps of this cycle that took the second pass
};

// Device-side state of one problem in a device-resident solve (the whole
// refinement loop in one graph launch): the decisions the host loop takes
// between cycles, taken by small kernels instead.
struct ResState {
  int open;          // needs another refinement step (a true residual)
  int inner;         // needs another inner cycle in this refinement step
  int result;        // vie_status of the problem (VIE_OK while running)
  int converged;
  int iters, outers, rounds, hist_len;
  int matvecs64, matvecs32, graph_cycles, reorth_steps;
  double target;     // absolute target of the next cycle
  double rel;        // last true relative residual
  double history[64];
};

// Everything a kernel needs about one problem.
struct ProbK {
  void* V;                 // (m + 1) basis vectors of the inner type
  void* Z;                 // m preconditioned vectors (== V without preconditioner)
  void* w;                 // one vector of the inner type
  size_t n;                // 3 nx ny nz
  const double2* b;        // right-hand side (complex128)
  double2* x64;            // iterate (complex128)
  double2* r64;            // residual (complex128)
  double2* y64;            // A x (complex128)
  double2* H;              // (m + 1) x m Hessenberg, column-major, ld = m + 1
  double2* hcol;           // CGS2 coefficients, pass 1 + pass 2
  double2* h2;             // pass-2 coefficients
  double2* g;              // rotated right-hand side of the least-squares problem
  double2* ysol;           // least-squares solution
  double* cs;
  double2* sn;
  double2* partial;        // (m + 2) x kDotBlocks partial sums
  double2* Q;              // product of the cycle's rotations, (m + 1) x (m + 1) row-major (cooperative step)
  SolveStatus* st;
  void* rin;               // inner residual (inner type): start of the next inner cycle
  void* d;                 // last cycle's correction Z y (inner type)
  double bnorm;            // ||b||
  double target;           // absolute target of the next cycle
  int from_inner;          // 1: the next cycle starts from rin, 0: from r64
  ResState* rs;            // device-resident solve: the problem's state (null in the host loop)
};

template <typename V> __device__ __forceinline__ double2 to_d2(V v) { return make_double2((double)v.x, (double)v.y); }
template <typename V> __device__ __forceinline__ V from_d2(double2 v);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }

// Arithmetic type of per-thread work on vectors of type V: complex64 vectors
// are multiplied and summed over a thread's few elements in FP32 (the FP64
// rate of this GPU is a small fraction of FP32), and every sum across threads
// and blocks is FP64.  complex128 vectors use FP64 throughout.
template <typename V> struct Acc;
template <> struct Acc<float2> { typedef float2 T; typedef float R; };
template <> struct Acc<double2> { typedef double2 T; typedef double R; };
template <typename A> __device__ __forceinline__ A zero_acc();
template <> __device__ __forceinline__ float2 zero_acc<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_acc<double2>() { return make_double2(0.0, 0.0); }
template <typename A> __device__ __forceinline__ A acc_from(double2 v);
template <> __device__ __forceinline__ float2 acc_from<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 acc_from<double2>(double2 v) { return v; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of `count` partials (the .x parts) by one block, fixed order; every
// thread gets the result.
__device__ double block_sum_partials(const double2* __restrict__ part, int count) {
  __shared__ double red[kThreads / 32];
  __shared__ double total;
  double t = 0.0;
  for (int b = threadIdx.x; b < count; b += blockDim.x) t += part[b].x;
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    total = s;
  }
  __syncthreads();
  return total;
}

template <typename R>
__device__ __forceinline__ void block_store_sum(R s, double2* out) {
  __shared__ double red[kThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *out = make_double2(t, 0.0);
  }
}

// Block b of a problem owns the element range [k0, k1) of length
// ceil(n / gridDim.x); the CGS2 kernels below share this decomposition so
// that the partial sums of one block can be formed right after its update.
struct Chunk {
  size_t k0, k1;
};
__device__ __forceinline__ Chunk chunk_of(size_t n) {
  const size_t c = (n + gridDim.x - 1) / gridDim.x;
  const size_t k0 = (size_t)blockIdx.x * c;
  return Chunk{k0 < n ? k0 : n, min(n, k0 + c)};
}

constexpr int kGroup = 8;   // basis vectors handled together (loads in flight per thread)

// Block-reduce kGroup complex sums and store them as partials of vectors
// i0 .. i0 + kGroup - 1 (those < nv).
// The warp-level part of the sum stays in the accumulator's precision (FP32
// for complex64: FP64 adds are slow on this GPU); warps are then combined in
// FP64.
template <typename A>
__device__ __forceinline__ void store_group(A (&acc)[kGroup], int i0, int nv, double2* __restrict__ partial,
                                            int nblk) {
  __shared__ double2 red[kThreads / 32][kGroup];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < kGroup; ++u) {
    acc[u].x = warp_sum(acc[u].x);
    acc[u].y = warp_sum(acc[u].y);
  }
  if (lane == 0)
#pragma unroll
    for (int u = 0; u < kGroup; ++u) red[warp][u] = make_double2((double)acc[u].x, (double)acc[u].y);
  __syncthreads();
  if (threadIdx.x < kGroup && i0 + threadIdx.x < nv) {
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t.x += red[w][threadIdx.x].x;
      t.y += red[w][threadIdx.x].y;
    }
    partial[(size_t)(i0 + threadIdx.x) * nblk + blockIdx.x] = t;
  }
  __syncthreads();
}

// partial[i * nblk + b] = sum over block b's chunk of conj(V_i[k]) w[k].
// grid (chunks, groups of kGroup vectors, problems): every block handles one
// chunk of elements for one group of vectors.
template <typename V>
__global__ void __launch_bounds__(kThreads) dots_kernel(const ProbK* __restrict__ P, int nv, int pass) {
  const ProbK& q = P[blockIdx.z];
  if (!q.st->active || (pass == 1 && !q.st->reorth)) return;
  const int i0 = blockIdx.y * kGroup;
  const V* __restrict__ Vb = (const V*)q.V;
  const V* __restrict__ w = (const V*)q.w;
  const size_t n = q.n;
  const Chunk ch = chunk_of(n);
  typedef typename Acc<V>::T A;
  A acc[kGroup];
#pragma unroll
  for (int u = 0; u < kGroup; ++u) acc[u] = zero_acc<A>();
  for (size_t k = ch.k0 + threadIdx.x; k < ch.k1; k += blockDim.x) {
    const V c = w[k];
    V a[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) a[u] = (i0 + u < nv) ? Vb[(size_t)(i0 + u) * n + k] : V{};
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      acc[u].x += a[u].x * c.x + a[u].y * c.y;
      acc[u].y += a[u].x * c.y - a[u].y * c.x;
    }
  }
  store_group(acc, i0, nv, q.partial, gridDim.x);
}

constexpr int kUpdGroup = 16;   // basis loads in flight per thread in the update

// w[k] -= sum_{i<nv} V_i[k] h[i], one element per thread, h = hcol (pass 0)
// or h2 (pass 1); pass 1 also writes the block's partial |w|^2 (Arnoldi norm).
template <typename V>
__global__ void __launch_bounds__(kThreads) update_kernel(const ProbK* __restrict__ P, int nv, int pass) {
  const ProbK& q = P[blockIdx.y];
  if (!q.st->active || (pass == 1 && !q.st->reorth)) return;
  typedef typename Acc<V>::T A;
  typedef typename Acc<V>::R AR;
  extern __shared__ unsigned char hs_raw[];
  A* hs = reinterpret_cast<A*>(hs_raw);
  const double2* h = pass == 0 ? q.hcol : q.h2;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = acc_from<A>(h[i]);
  __syncthreads();
  const V* __restrict__ Vb = (const V*)q.V;
  V* __restrict__ w = (V*)q.w;
  const size_t n = q.n;
  AR nrm = 0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const V w0 = w[k];
    A acc;
    acc.x = w0.x;
    acc.y = w0.y;
    for (int i0 = 0; i0 < nv; i0 += kUpdGroup) {
      V a[kUpdGroup];
#pragma unroll
      for (int u = 0; u < kUpdGroup; ++u) a[u] = (i0 + u < nv) ? Vb[(size_t)(i0 + u) * n + k] : V{};
#pragma unroll
      for (int u = 0; u < kUpdGroup; ++u) {
        if (i0 + u < nv) {
          acc.x -= a[u].x * hs[i0 + u].x - a[u].y * hs[i0 + u].y;
          acc.y -= a[u].x * hs[i0 + u].y + a[u].y * hs[i0 + u].x;
        }
      }
    }
    V out;
    out.x = acc.x;
    out.y = acc.y;
    w[k] = out;
    nrm += out.x * out.x + out.y * out.y;
  }
  block_store_sum(nrm, q.partial + blockIdx.x);
}

// After the first pass: ||w'||^2 from the update's partials and ||h1||^2 from
// the coefficients; the second pass is needed when ||w'||^2 < (||w'||^2 +
// ||h1||^2) / 2, i.e. ||w'|| < ||w|| / sqrt 2 (||w||^2 = ||w'||^2 + ||h1||^2 for an
// orthonormal basis).  One block per problem.
__global__ void __launch_bounds__(kThreads) reorth_decide_kernel(const ProbK* __restrict__ P, int nblk, int nv) {
  const ProbK& q = P[blockIdx.x];
  if (!q.st->active) return;
  const double w2 = block_sum_partials(q.partial, nblk);
  if (threadIdx.x == 0) {
    double h2 = 0.0;
    for (int i = 0; i < nv; ++i) h2 += q.hcol[i].x * q.hcol[i].x + q.hcol[i].y * q.hcol[i].y;
    const int r = (w2 < 0.5 * (w2 + h2)) ? 1 : 0;
    q.st->reorth = r;
    q.st->reorth_count += r;
  }
}

// pass 0: hcol[i] = sum_b partial; pass 1: h2[i] = sum_b partial, hcol[i] += h2[i].
// Fixed summation order (deterministic).  grid (nv, problems).
__global__ void __launch_bounds__(kThreads) reduce_partials_kernel(const ProbK* __restrict__ P, int nblk, int pass) {
  const ProbK& q = P[blockIdx.y];
  if (!q.st->active || (pass == 1 && !q.st->reorth)) return;
  const int i = blockIdx.x;
  __shared__ double sre[kThreads], sim[kThreads];
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    re += q.partial[(size_t)i * nblk + b].x;
    im += q.partial[(size_t)i * nblk + b].y;
  }
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int t = blockDim.x / 2; t > 0; t >>= 1) {
    if (threadIdx.x < t) {
      sre[threadIdx.x] += sre[threadIdx.x + t];
      sim[threadIdx.x] += sim[threadIdx.x + t];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (pass == 0) {
      q.hcol[i] = make_double2(sre[0], sim[0]);
    } else {
      q.h2[i] = make_double2(sre[0], sim[0]);
      q.hcol[i].x += sre[0];
      q.hcol[i].y += sim[0];
    }
  }
}

// partial[b] = sum |b[k]|^2 (used before any cycle: no status check)
__global__ void __launch_bounds__(kThreads) norm2_b_kernel(const ProbK* __restrict__ P) {
  const ProbK& q = P[blockIdx.y];
  double s = 0.0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < q.n; k += (size_t)gridDim.x * blockDim.x) {
    const double2 a = q.b[k];
    s += a.x * a.x + a.y * a.y;
  }
  block_store_sum(s, q.partial + blockIdx.x);
}

// r = b - y (complex128) with norm partials of r
__global__ void __launch_bounds__(kThreads) residual_kernel(const ProbK* __restrict__ P) {
  const ProbK& q = P[blockIdx.y];
  if (q.rs && !q.rs->open) return;
  double s = 0.0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < q.n; k += (size_t)gridDim.x * blockDim.x) {
    const double2 v = make_double2(q.b[k].x - q.y64[k].x, q.b[k].y - q.y64[k].y);
    q.r64[k] = v;
    s += v.x * v.x + v.y * v.y;
  }
  block_store_sum(s, q.partial + blockIdx.x);
}

// One block per problem: beta = ||r|| from the residual partials, status and g.
__global__ void __launch_bounds__(kThreads) init_cycle_kernel(const ProbK* __restrict__ P, int nblk, int m) {
  const ProbK& q = P[blockIdx.x];
  if (q.rs && !q.rs->inner) {
    // device-resident solve: this problem takes no cycle now
    if (threadIdx.x == 0) {
      SolveStatus* st = q.st;
      st->active = 0;
      st->j = 0;
      st->converged = 0;
      st->breakdown = 0;
      st->reorth_count = 0;
    }
    return;
  }
  const double beta = sqrt(block_sum_partials(q.partial, nblk));
  for (int i = threadIdx.x; i <= m; i += blockDim.x) q.g[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
  if (threadIdx.x == 0) {
    SolveStatus* st = q.st;
    st->active = (beta > 0.0 && isfinite(beta)) ? 1 : 0;
    st->j = 0;
    st->converged = 0;
    st->breakdown = isfinite(beta) ? 0 : 1;
    st->beta = beta;
    st->target = q.rs ? q.rs->target : q.target;
    st->resid = beta;
    st->inv_h = beta > 0.0 ? 1.0 / beta : 0.0;
    st->reorth_count = 0;
  }
}

// V_0 = r / beta  (converted to the inner type)
template <typename V>
__global__ void __launch_bounds__(kThreads) start_vector_kernel(const ProbK* __restrict__ P) {
  const ProbK& q = P[blockIdx.y];
  if (!q.st->active) return;
  const double s = q.st->inv_h;
  V* __restrict__ v0 = (V*)q.V;
  const V* __restrict__ rin = (const V*)q.rin;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < q.n; k += (size_t)gridDim.x * blockDim.x) {
    const double2 a = q.from_inner ? to_d2(rin[k]) : q.r64[k];
    v0[k] = from_d2<V>(make_double2(a.x * s, a.y * s));
  }
}

// rin = r64 (converted to the inner type), norm partials of rin
template <typename V>
__global__ void __launch_bounds__(kThreads) inner_from_outer_kernel(const ProbK* __restrict__ P) {
  const ProbK& q = P[blockIdx.y];
  if (q.rs && !q.rs->inner) return;
  V* __restrict__ rin = (V*)q.rin;
  double s = 0.0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < q.n; k += (size_t)gridDim.x * blockDim.x) {
    const V v = from_d2<V>(q.r64[k]);
    rin[k] = v;
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  block_store_sum(s, q.partial + blockIdx.x);
}

// rin -= w (w = A d from the inner operator), norm partials of rin
template <typename V>
__global__ void __launch_bounds__(kThreads) inner_residual_kernel(const ProbK* __restrict__ P) {
  const ProbK& q = P[blockIdx.y];
  if (q.rs && !q.rs->inner) return;
  V* __restrict__ rin = (V*)q.rin;
  const V* __restrict__ ad = (const V*)q.w;
  typename Acc<V>::R s = 0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < q.n; k += (size_t)gridDim.x * blockDim.x) {
    V r = rin[k];
    const V a = ad[k];
    r.x -= a.x;
    r.y -= a.y;
    rin[k] = r;
    s += r.x * r.x + r.y * r.y;
  }
  block_store_sum(s, q.partial + blockIdx.x);
}

// One block per problem: h_{j+1,j} = ||w|| (parallel reduction), then thread 0
// applies the previous rotations to column j in shared memory, forms the new
// rotation and updates g and the status; the column goes back to H.
__global__ void __launch_bounds__(kThreads) arnoldi_step_kernel(const ProbK* __restrict__ P, int nblk, int ldh,
                                                               int j) {
  const ProbK& q = P[blockIdx.x];
  SolveStatus* st = q.st;
  if (!st->active) return;
  __shared__ double2 col[kMaxRestart + 1];
  __shared__ double csh[kMaxRestart];
  __shared__ double2 snh[kMaxRestart];
  const double hn = sqrt(block_sum_partials(q.partial, nblk));
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = q.hcol[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    csh[i] = q.cs[i];
    snh[i] = q.sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    col[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
      const double c = csh[i];
      const double2 s = snh[i];
      const double2 a = col[i], b = col[i + 1];
      // t = c a + s b ; b' = -conj(s) a + c b
      col[i] = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
      col[i + 1] = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    }
    const double2 a = col[j], b = col[j + 1];
    const double aa = hypot(a.x, a.y), ab = hypot(b.x, b.y);
    const double den = hypot(aa, ab);
    double c;
    double2 s;
    if (den == 0.0) {
      c = 1.0; s = make_double2(0.0, 0.0);
    } else if (aa == 0.0) {
      c = 0.0; s = make_double2(1.0, 0.0);
    } else {
      c = aa / den;
      const double2 ua = make_double2(a.x / aa, a.y / aa);   // s = (a/|a|) conj(b) / den
      s = make_double2((ua.x * b.x + ua.y * b.y) / den, (ua.y * b.x - ua.x * b.y) / den);
    }
    q.cs[j] = c;
    q.sn[j] = s;
    col[j] = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
    col[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = q.g[j];
    const double2 g1 = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    q.g[j + 1] = g1;
    q.g[j] = make_double2(c * gj.x, c * gj.y);
    const double res = hypot(g1.x, g1.y);
    st->j = j + 1;
    st->resid = res;
    if (!(isfinite(hn) && isfinite(res))) {
      st->breakdown = 1;
      st->active = 0;
      st->j = j;          // drop the non-finite column
    } else {
      if (res <= st->target) {
        st->converged = 1;
        st->active = 0;
      }
      if (hn <= 1e-300 || hn <= 1e-14 * st->beta) {
        st->breakdown = 1;
        st->active = 0;
      }
      st->inv_h = (hn > 0.0) ? 1.0 / hn : 0.0;
    }
  }
  __syncthreads();
  double2* H = q.H + (size_t)j * ldh;
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) H[i] = col[i];
}

// v_{j+1} = w / h_{j+1,j}
template <typename V>
__global__ void __launch_bounds__(kThreads) next_vector_kernel(const ProbK* __restrict__ P, int j) {
  const ProbK& q = P[blockIdx.y];
  if (!q.st->active) return;
  const typename Acc<V>::R s = (typename Acc<V>::R)q.st->inv_h;
  const V* __restrict__ w = (const V*)q.w;
  V* __restrict__ v = (V*)q.V + (size_t)(j + 1) * q.n;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < q.n; k += (size_t)gridDim.x * blockDim.x) {
    V a = w[k];
    a.x *= s;
    a.y *= s;
    v[k] = a;
  }
}

// Back substitution R y = g over the st->j columns, one block per problem.
__global__ void __launch_bounds__(kThreads) backsolve_kernel(const ProbK* __restrict__ P, int ldh) {
  const ProbK& q = P[blockIdx.x];
  const int m = q.st->j;
  __shared__ double2 ys[kMaxRestart];
  for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = q.g[i];
  __syncthreads();
  for (int i = m - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      const double2 r = q.H[(size_t)i * ldh + i];
      const double2 v = ys[i];
      const double d = r.x * r.x + r.y * r.y;
      ys[i] = make_double2((v.x * r.x + v.y * r.y) / d, (v.y * r.x - v.x * r.y) / d);
    }
    __syncthreads();
    const double2 yi = ys[i];
    for (int k = threadIdx.x; k < i; k += blockDim.x) {
      const double2 r = q.H[(size_t)i * ldh + k];
      ys[k].x -= r.x * yi.x - r.y * yi.y;
      ys[k].y -= r.x * yi.y + r.y * yi.x;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) q.ysol[i] = ys[i];
}

// x[k] += sum_{i < st->j} Z_i[k] y_i  (x complex128, FP64 accumulation)
template <typename V>
__global__ void __launch_bounds__(kThreads) update_x_kernel(const ProbK* __restrict__ P) {
  const ProbK& q = P[blockIdx.y];
  const int m = q.st->j;
  if (m == 0) return;
  // the correction Z y is summed in the vector's precision (complex64: it only
  // has to meet the loose inner tolerance); x itself accumulates in FP64
  typedef typename Acc<V>::T A;
  extern __shared__ unsigned char ys_raw[];
  A* ys = reinterpret_cast<A*>(ys_raw);
  for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = acc_from<A>(q.ysol[i]);
  __syncthreads();
  const V* __restrict__ Zb = (const V*)q.Z;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < q.n; k += (size_t)gridDim.x * blockDim.x) {
    A acc = zero_acc<A>();
    for (int i = 0; i < m; ++i) {
      const V z = Zb[(size_t)i * q.n + k];
      acc.x += z.x * ys[i].x - z.y * ys[i].y;
      acc.y += z.x * ys[i].y + z.y * ys[i].x;
    }
    q.x64[k].x += (double)acc.x;
    q.x64[k].y += (double)acc.y;
    if (q.d) {
      V dv;
      dv.x = acc.x;
      dv.y = acc.y;
      ((V*)q.d)[k] = dv;
    }
  }
}

// ---------------------------------------------------------------------------
// The whole Gram-Schmidt step in one cooperative launch
// ---------------------------------------------------------------------------
// One block of 512 threads per SM (all resident: cooperative launch); the
// phases of a step are separated by a grid barrier instead of kernel
// boundaries:
//   dots (pass 1) | reduce -> h1 | w -= V h1, |w'|^2 | decide second pass
//   [ dots (pass 2) | reduce -> h2, h1 + h2 | w -= V h2, |w''|^2 ] |
//   h_{j+1,j}, v_{j+1} = w / h_{j+1,j}, Givens step (one block per problem)
// with the same element chunks, partial sums and fixed summation orders as
// the separate kernels above (the decision and ||w|| are computed
// identically by every block).  Every barrier wait is bounded: a block that
// waited kBarrierCycles sets the abort word and every block returns.  Values
// another block wrote in this launch (partials, coefficients) are read with
// ld.global.cg, past the SM's L1.
constexpr int kCoopThreadsMax = 1024;
// threads per block of the cooperative step (up to 128 registers: the
// complex64 dots keep all coefficients of a step in registers)
template <typename V> constexpr int coop_threads() { return 512; }
constexpr int kCoopDotsMax = 32;   // complex64 dots with all vectors in one sweep up to this basis size
// Batches of more problems take the separate kernels, whose launches carry
// one grid plane per problem (measured on the 48 uneven guides: 5.61 s with
// the separate kernels, 5.84 s with every block looping over the 48 problems
// in each phase of the cooperative step).
constexpr int kCoopMaxProblems = 8;
constexpr long long kBarrierCycles = 2000000000LL;   // ~1 s

// bar[0] arrivals, bar[1] generation, bar[2] abort (a wait gave up after
// `limit` SM clocks)
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, long long limit = kBarrierCycles) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* vabort = bar + 2;
    const unsigned g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*vabort) { ok = 0; break; }
        if (clock64() - t0 > limit) { atomicExch(bar + 2, 1u); ok = 0; break; }
      }
    }
    __threadfence();
    ok_s = ok && !*vabort;
  }
  __syncthreads();
  return ok_s != 0;
}

// kGroup complex sums of the block -> partial[(i0 + u) * nblk + blockIdx.x]
template <typename A>
__device__ __forceinline__ void coop_store_group(A (&acc)[kGroup], int i0, int nv, double2* __restrict__ partial,
                                                 int nblk) {
  __shared__ double2 red[kCoopThreadsMax / 32][kGroup];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < kGroup; ++u) {
    acc[u].x = warp_sum(acc[u].x);
    acc[u].y = warp_sum(acc[u].y);
  }
  if (lane == 0)
#pragma unroll
    for (int u = 0; u < kGroup; ++u) red[warp][u] = make_double2((double)acc[u].x, (double)acc[u].y);
  __syncthreads();
  if (threadIdx.x < kGroup && i0 + threadIdx.x < nv) {
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t.x += red[w][threadIdx.x].x;
      t.y += red[w][threadIdx.x].y;
    }
    partial[(size_t)(i0 + threadIdx.x) * nblk + blockIdx.x] = t;
  }
  __syncthreads();
}

// dots of the block's chunk with vectors 0 .. nv-1 -> partial slots 0 .. nv-1.
// Complex64 with nv <= kCoopDotsMax: one sweep over the chunk, w[k] read once
// and all nv products accumulated in registers (like the update); otherwise
// kGroup vectors per sweep.
template <typename V>
__device__ void coop_dots(const ProbK& q, int nv, int nblk) {
  typedef typename Acc<V>::T A;
  const V* __restrict__ Vb = (const V*)q.V;
  const V* __restrict__ w = (const V*)q.w;
  const size_t n = q.n;
  const Chunk ch = chunk_of(n);
  if constexpr (sizeof(V) == sizeof(float2)) {
    if (nv <= kCoopDotsMax) {
      A acc[kCoopDotsMax];
#pragma unroll
      for (int u = 0; u < kCoopDotsMax; ++u) acc[u] = zero_acc<A>();
      // two elements per iteration (k, k + blockDim): twice the loads in flight
      for (size_t k = ch.k0 + threadIdx.x; k < ch.k1; k += 2 * (size_t)blockDim.x) {
        const size_t k2 = k + blockDim.x;
        const bool two = k2 < ch.k1;
        const V c = w[k];
        const V c2 = two ? w[k2] : V{};
#pragma unroll
        for (int i0 = 0; i0 < kCoopDotsMax; i0 += kGroup) {
          if (i0 < nv) {
            V a[kGroup], b[kGroup];
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
              a[u] = (i0 + u < nv) ? Vb[(size_t)(i0 + u) * n + k] : V{};
              b[u] = (two && i0 + u < nv) ? Vb[(size_t)(i0 + u) * n + k2] : V{};
            }
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
              acc[i0 + u].x += a[u].x * c.x + a[u].y * c.y + b[u].x * c2.x + b[u].y * c2.y;
              acc[i0 + u].y += a[u].x * c.y - a[u].y * c.x + b[u].x * c2.y - b[u].y * c2.x;
            }
          }
        }
      }
#pragma unroll
      for (int i0 = 0; i0 < kCoopDotsMax; i0 += kGroup) {
        if (i0 < nv) {
          A grp[kGroup];
#pragma unroll
          for (int u = 0; u < kGroup; ++u) grp[u] = acc[i0 + u];
          coop_store_group(grp, i0, nv, q.partial, nblk);
        }
      }
      return;
    }
  }
  for (int i0 = 0; i0 < nv; i0 += kGroup) {
    A acc[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) acc[u] = zero_acc<A>();
    for (size_t k = ch.k0 + threadIdx.x; k < ch.k1; k += blockDim.x) {
      const V c = w[k];
      V a[kGroup];
#pragma unroll
      for (int u = 0; u < kGroup; ++u) a[u] = (i0 + u < nv) ? Vb[(size_t)(i0 + u) * n + k] : V{};
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        acc[u].x += a[u].x * c.x + a[u].y * c.y;
        acc[u].y += a[u].x * c.y - a[u].y * c.x;
      }
    }
    coop_store_group(acc, i0, nv, q.partial, nblk);
  }
}

// sum of partial[slot * nblk + 0 .. nblk) by one warp in a fixed order
__device__ __forceinline__ double2 warp_sum_partials(const double2* __restrict__ part, int nblk) {
  const int lane = threadIdx.x & 31;
  double2 t = make_double2(0.0, 0.0);
  for (int b0 = 0; b0 < nblk; b0 += 8 * 32) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * 32 + lane;
      v[u] = b < nblk ? __ldcg(part + b) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      t.x += v[u].x;
      t.y += v[u].y;
    }
  }
  t.x = warp_sum(t.x);
  t.y = warp_sum(t.y);
  t.x = __shfl_sync(0xffffffffu, t.x, 0);
  t.y = __shfl_sync(0xffffffffu, t.y, 0);
  return t;
}

// w -= V h over the block's chunk (h: nv coefficients in shared memory), |w|^2
// of the chunk -> partial[slot * nblk + blockIdx.x]
template <typename V>
__device__ void coop_update(const ProbK& q, int nv, const typename Acc<V>::T* hs, int slot, int nblk) {
  typedef typename Acc<V>::T A;
  typedef typename Acc<V>::R AR;
  const V* __restrict__ Vb = (const V*)q.V;
  V* __restrict__ w = (V*)q.w;
  const size_t n = q.n;
  const Chunk ch = chunk_of(n);
  AR nrm = 0;
  // complex64: two elements per iteration (k, k + blockDim), twice the loads
  // in flight; complex128 (registers) one
  constexpr int E = sizeof(V) == sizeof(float2) ? 2 : 1;
  for (size_t k = ch.k0 + threadIdx.x; k < ch.k1; k += E * (size_t)blockDim.x) {
    const size_t k2 = k + blockDim.x;
    const bool two = E == 2 && k2 < ch.k1;
    const V w0 = w[k];
    const V w1 = two ? w[k2] : V{};
    A acc, acc2;
    acc.x = w0.x;
    acc.y = w0.y;
    acc2.x = w1.x;
    acc2.y = w1.y;
    for (int i0 = 0; i0 < nv; i0 += kUpdGroup) {
      V a[kUpdGroup], b[E == 2 ? kUpdGroup : 1];
#pragma unroll
      for (int u = 0; u < kUpdGroup; ++u) {
        a[u] = (i0 + u < nv) ? Vb[(size_t)(i0 + u) * n + k] : V{};
        if constexpr (E == 2) b[u] = (two && i0 + u < nv) ? Vb[(size_t)(i0 + u) * n + k2] : V{};
      }
#pragma unroll
      for (int u = 0; u < kUpdGroup; ++u) {
        if (i0 + u < nv) {
          const A h = hs[i0 + u];
          acc.x -= a[u].x * h.x - a[u].y * h.y;
          acc.y -= a[u].x * h.y + a[u].y * h.x;
          if constexpr (E == 2) {
            acc2.x -= b[u].x * h.x - b[u].y * h.y;
            acc2.y -= b[u].x * h.y + b[u].y * h.x;
          }
        }
      }
    }
    V out;
    out.x = acc.x;
    out.y = acc.y;
    w[k] = out;
    nrm += out.x * out.x + out.y * out.y;
    if (two) {
      V out2;
      out2.x = acc2.x;
      out2.y = acc2.y;
      w[k2] = out2;
      nrm += out2.x * out2.x + out2.y * out2.y;
    }
  }
  __shared__ double red[kCoopThreadsMax / 32];
  AR t = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) u += red[i];
    q.partial[(size_t)slot * nblk + blockIdx.x] = make_double2(u, 0.0);
  }
  __syncthreads();
}

// pairs (problem, vector) distributed over the warps of the grid: coefficient
// = sum of that vector's partials; pass 0 writes hcol, pass 1 h2 and hcol += h2
__device__ void coop_reduce(const ProbK* __restrict__ P, int count, const int* sel, int nv, int nblk, int pass) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int pairs = count * nv;
  for (int pi = blockIdx.x * wpb + warp; pi < pairs; pi += gridDim.x * wpb) {
    const int p = pi / nv, i = pi - p * nv;
    if (!sel[p]) continue;
    const ProbK& q = P[p];
    const double2 t = warp_sum_partials(q.partial + (size_t)i * nblk, nblk);
    if (lane == 0) {
      if (pass == 0) {
        q.hcol[i] = t;
      } else {
        const double2 h1 = __ldcg(q.hcol + i);
        q.h2[i] = t;
        q.hcol[i] = make_double2(h1.x + t.x, h1.y + t.y);
      }
    }
  }
}

// The FP64 least-squares step of problem q for column j by the block that
// owns q.  The rotations of the cycle are kept multiplied out, Q = O_{j-1}
// ... O_0 ((j + 1) x (j + 1), row-major, ld = m + 1 = ldh), so that applying
// them to the new column is a matrix-vector product (a warp per row, lanes
// over the columns, fixed-order reduction) instead of a chain of j
// dependent rotations; thread 0 then forms the new rotation O_j on
// (r_j, h_{j+1,j}), updates g and the status, and Q's rows j and j + 1 are
// replaced by O_j applied to (row j, e_{j+1}).  sh: j + 2 double2.
__device__ void coop_givens(const ProbK& q, int j, int ldh, double hn, double inv, double2* sh) {
  double2* r = sh;
  __shared__ double2 rot[2];   // (c, 0), s
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int ldq = ldh;
  __syncthreads();
  for (int i = warp; i <= j; i += nw) {
    double re = 0.0, im = 0.0;
    for (int k = lane; k <= j; k += 32) {
      const double2 g = j == 0 ? make_double2(1.0, 0.0) : q.Q[(size_t)i * ldq + k];
      const double2 h = __ldcg(q.hcol + k);
      re += g.x * h.x - g.y * h.y;
      im += g.x * h.y + g.y * h.x;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) r[i] = make_double2(re, im);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SolveStatus* st = q.st;
    const double2 a = r[j], b = make_double2(hn, 0.0);
    const double aa = hypot(a.x, a.y), ab = hypot(b.x, b.y);
    const double den = hypot(aa, ab);
    double c;
    double2 s;
    if (den == 0.0) {
      c = 1.0; s = make_double2(0.0, 0.0);
    } else if (aa == 0.0) {
      c = 0.0; s = make_double2(1.0, 0.0);
    } else {
      c = aa / den;
      const double2 ua = make_double2(a.x / aa, a.y / aa);
      s = make_double2((ua.x * b.x + ua.y * b.y) / den, (ua.y * b.x - ua.x * b.y) / den);
    }
    q.cs[j] = c;
    q.sn[j] = s;
    rot[0] = make_double2(c, 0.0);
    rot[1] = s;
    r[j] = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
    r[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = q.g[j];
    const double2 g1 = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    q.g[j + 1] = g1;
    q.g[j] = make_double2(c * gj.x, c * gj.y);
    const double res = hypot(g1.x, g1.y);
    st->j = j + 1;
    st->resid = res;
    if (!(isfinite(hn) && isfinite(res))) {
      st->breakdown = 1;
      st->active = 0;
      st->j = j;
    } else {
      if (res <= st->target) {
        st->converged = 1;
        st->active = 0;
      }
      if (hn <= 1e-300 || hn <= 1e-14 * st->beta) {
        st->breakdown = 1;
        st->active = 0;
      }
      st->inv_h = inv;
    }
  }
  __syncthreads();
  double2* H = q.H + (size_t)j * ldh;
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) H[i] = r[i];
  // Q <- O_j diag(Q, 1): rows j and j + 1 over columns 0 .. j + 1; column
  // j + 1 of the rows above is zero
  const double c = rot[0].x;
  const double2 s = rot[1];
  for (int k = threadIdx.x; k <= j + 1; k += blockDim.x) {
    double2 gj;
    if (k == j + 1) gj = make_double2(0.0, 0.0);
    else if (j == 0) gj = make_double2(k == 0 ? 1.0 : 0.0, 0.0);
    else gj = q.Q[(size_t)j * ldq + k];
    const double2 e = make_double2(k == j + 1 ? 1.0 : 0.0, 0.0);
    // row j' = c gj + s e ; row j+1' = -conj(s) gj + c e
    q.Q[(size_t)j * ldq + k] = make_double2(c * gj.x + (s.x * e.x - s.y * e.y), c * gj.y + (s.x * e.y + s.y * e.x));
    q.Q[(size_t)(j + 1) * ldq + k] =
        make_double2(-(s.x * gj.x + s.y * gj.y) + c * e.x, -(s.x * gj.y - s.y * gj.x) + c * e.y);
  }
  for (int i = threadIdx.x; i < j; i += blockDim.x) q.Q[(size_t)i * ldq + j + 1] = make_double2(0.0, 0.0);
}

// Step j (nv = j + 1 basis vectors) for the count problems of P after the
// operator has written w; with set_next, the last block to finish also sets
// the condition `next` of the following step's graph node.  Dynamic shared
// memory: nv coefficients, then (j + 2) + j double2 and j double for the
// Givens step.
template <typename V>
__global__ void __launch_bounds__(coop_threads<V>(), 1) arnoldi_coop_kernel(const ProbK* __restrict__ P, int count,
                                                                      int nv, int ldh, unsigned* bar,
                                                                      cudaGraphConditionalHandle next, int set_next) {
  typedef typename Acc<V>::T A;
  const int j = nv - 1;
  const int nblk = gridDim.x;
  const unsigned nb = gridDim.x;
  __shared__ int act[kCoopMaxProblems], reo[kCoopMaxProblems];
  __shared__ double hn_s[kCoopMaxProblems];
  __shared__ int any_reo;
  extern __shared__ unsigned char coop_raw[];
  A* hs = reinterpret_cast<A*>(coop_raw);                                   // nv coefficients
  double2* col = reinterpret_cast<double2*>(coop_raw + ((nv * sizeof(A) + 15) / 16) * 16);
  for (int p = threadIdx.x; p < count; p += blockDim.x) act[p] = P[p].st->active;
  __syncthreads();
  // dots, pass 1
  for (int p = 0; p < count; ++p)
    if (act[p]) coop_dots<V>(P[p], nv, nblk);
  if (!grid_barrier(bar, nb)) return;
  coop_reduce(P, count, act, nv, nblk, 0);
  if (!grid_barrier(bar, nb)) return;
  for (int p = 0; p < count; ++p) {
    if (!act[p]) continue;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = acc_from<A>(__ldcg(P[p].hcol + i));
    __syncthreads();
    coop_update<V>(P[p], nv, hs, nv, nblk);
  }
  if (!grid_barrier(bar, nb)) return;
  // second-pass decision (identical in every block): ||w'||^2 < (||w'||^2 + ||h1||^2) / 2
  if (threadIdx.x < 32) {
    int any = 0;
    for (int p = 0; p < count; ++p) {
      int r = 0;
      if (act[p]) {
        const ProbK& q = P[p];
        const double w2 = warp_sum_partials(q.partial + (size_t)nv * nblk, nblk).x;
        double h2 = 0.0;
        for (int i = threadIdx.x; i < nv; i += 32) {
          const double2 h = __ldcg(q.hcol + i);
          h2 += h.x * h.x + h.y * h.y;
        }
        h2 = warp_sum(h2);
        h2 = __shfl_sync(0xffffffffu, h2, 0);
        r = (w2 < 0.5 * (w2 + h2)) ? 1 : 0;
        if (threadIdx.x == 0 && blockIdx.x == 0) {
          q.st->reorth = r;
          q.st->reorth_count += r;
        }
      }
      if (threadIdx.x == 0) reo[p] = r;
      any |= r;
    }
    if (threadIdx.x == 0) any_reo = any;
  }
  __syncthreads();
  if (any_reo) {
    for (int p = 0; p < count; ++p)
      if (reo[p]) coop_dots<V>(P[p], nv, nblk);
    if (!grid_barrier(bar, nb)) return;
    coop_reduce(P, count, reo, nv, nblk, 1);
    if (!grid_barrier(bar, nb)) return;
    for (int p = 0; p < count; ++p) {
      if (!reo[p]) continue;
      for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = acc_from<A>(__ldcg(P[p].h2 + i));
      __syncthreads();
      coop_update<V>(P[p], nv, hs, nv + 1, nblk);
    }
    if (!grid_barrier(bar, nb)) return;
  }
  // h_{j+1,j} = ||w|| (same order in every block), v_{j+1}, Givens step
  if (threadIdx.x < 32)
    for (int p = 0; p < count; ++p)
      if (act[p]) {
        const double t = warp_sum_partials(P[p].partial + (size_t)(reo[p] ? nv + 1 : nv) * nblk, nblk).x;
        if (threadIdx.x == 0) hn_s[p] = sqrt(t);
      }
  __syncthreads();
  for (int p = 0; p < count; ++p) {
    if (!act[p]) continue;
    const ProbK& q = P[p];
    const double hn = hn_s[p];
    const double inv = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
    const typename Acc<V>::R sc = (typename Acc<V>::R)inv;
    const V* __restrict__ w = (const V*)q.w;
    V* __restrict__ v = (V*)q.V + (size_t)(j + 1) * q.n;
    const Chunk ch = chunk_of(q.n);
    for (size_t k = ch.k0 + threadIdx.x; k < ch.k1; k += blockDim.x) {
      V a = w[k];
      a.x *= sc;
      a.y *= sc;
      v[k] = a;
    }
    if (blockIdx.x == (unsigned)(p % nblk)) coop_givens(q, j, ldh, hn, inv, col);
  }
  if (set_next) {
    // the last block to finish (ticket in bar[3]) sets the condition of the
    // next step's graph node: 1 while any problem is still active
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(bar + 3, 1u) == nb - 1) {
        __threadfence();
        int any = 0;
        for (int p = 0; p < count; ++p) any |= __ldcg(&P[p].st->active);
        cudaGraphSetConditional(next, any ? 1u : 0u);
        atomicExch(bar + 3, 0u);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Device-resident solve: the decisions between cycles as kernels
// ---------------------------------------------------------------------------
// Control block of a device-resident solve: the time limit (globaltimer) and
// the iteration counters of its two loops, which bound them whatever the
// per-problem state says.
struct ResCtl {
  unsigned long long t0;        // globaltimer at the first outer step
  unsigned long long limit_ns;  // time limit of the solve
  int outer_iters;              // outer-loop iterations run
  int cap_outer;                // at most this many
  int inner_iters;              // inner-loop iterations in the current outer step
  int pad;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One block per problem, after the true residual r = b - A x of the open
// problems: beta = ||r||, the relative residual and its history, then the
// outcome of the problem (converged, non-finite, caps, time limit) or the
// target of the next inner cycles (the host loop's refinement step).
__global__ void __launch_bounds__(kThreads) outer_decide_kernel(const ProbK* __restrict__ P, int nblk, double tol,
                                                               double inner_tol, int mixed, int max_iters,
                                                               int max_outer, ResCtl* ctl) {
  const ProbK& q = P[blockIdx.x];
  ResState* rs = q.rs;
  __shared__ int open;
  if (threadIdx.x == 0) {
    open = rs->open;
    if (!open) rs->inner = 0;
  }
  __syncthreads();
  if (!open) return;
  const double beta = sqrt(block_sum_partials(q.partial, nblk));
  if (threadIdx.x != 0) return;
  if (ctl->t0 == 0ull) atomicCAS(&ctl->t0, 0ull, global_ns());
  rs->matvecs64++;
  const double rel = beta / q.bnorm;
  rs->rel = rel;
  if (rs->outers < 64) rs->history[rs->outers] = rel;
  rs->hist_len = rs->outers + 1 < 64 ? rs->outers + 1 : 64;
  rs->inner = 0;
  if (!isfinite(beta)) {
    rs->result = VIE_ERR_NONFINITE;
    rs->open = 0;
  } else if (beta <= tol * q.bnorm) {
    rs->converged = 1;
    rs->open = 0;
  } else if (rs->iters >= max_iters || rs->outers >= max_outer) {
    rs->result = VIE_ERR_NOT_CONVERGED;
    rs->open = 0;
  } else if (global_ns() - ctl->t0 > ctl->limit_ns) {
    rs->result = VIE_ERR_TIMEOUT;
    rs->open = 0;
  } else {
    // plain mode goes for tol ||b||; mixed asks the complex64 cycles for a
    // reduction inner_tol, never below half the outer target
    rs->target = mixed ? fmax(inner_tol * beta, 0.5 * tol * q.bnorm) : tol * q.bnorm;
    rs->inner = 1;
    rs->rounds = 0;
  }
}

// any problem with an inner cycle to run: the inner loop's condition
__global__ void outer_finalize_kernel(const ProbK* __restrict__ P, int count, ResCtl* ctl,
                                      cudaGraphConditionalHandle h_in) {
  int any = 0;
  for (int p = threadIdx.x; p < count; p += blockDim.x) any |= P[p].rs->inner;
  any = __any_sync(0xffffffffu, any);
  if (threadIdx.x == 0) {
    ctl->inner_iters = 0;
    cudaGraphSetConditional(h_in, any ? 1u : 0u);
  }
}

// the steps of the next cycle: step 0 runs, the later ones as the steps set them
__global__ void reset_steps_kernel(const cudaGraphConditionalHandle* __restrict__ h, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) cudaGraphSetConditional(h[k], k == 0 ? 1u : 0u);
}

// After a cycle (one warp): step counts, the outcome of the cycle, and whether
// the problem takes another inner cycle (mixed mode) or the next true
// residual; the inner loop's condition.
__global__ void inner_decide_kernel(const ProbK* __restrict__ P, int count, int mixed, int max_iters, ResCtl* ctl,
                                    cudaGraphConditionalHandle h_in) {
  int any = 0;
  for (int p = threadIdx.x; p < count; p += blockDim.x) {
    ResState* rs = P[p].rs;
    if (!rs->inner) continue;
    const SolveStatus* st = P[p].st;
    const int steps = st->j;
    rs->iters += steps;
    if (mixed) rs->matvecs32 += steps; else rs->matvecs64 += steps;
    rs->graph_cycles += 1;
    rs->reorth_steps += st->reorth_count;
    if (steps == 0) {
      rs->result = VIE_ERR_NOT_CONVERGED;
      rs->open = 0;
      rs->inner = 0;
      continue;
    }
    const bool more = mixed && !st->converged && !st->breakdown && rs->rounds + 1 < kMaxInnerCycles &&
                      rs->iters < max_iters;
    rs->rounds += 1;
    if (more) {
      rs->matvecs32 += 1;      // A d for the inner residual
      any = 1;
    } else {
      rs->inner = 0;
      rs->outers += 1;
    }
  }
  any = __any_sync(0xffffffffu, any);
  if (threadIdx.x == 0) {
    ctl->inner_iters += 1;
    cudaGraphSetConditional(h_in, (any && ctl->inner_iters < kMaxInnerCycles) ? 1u : 0u);
  }
}

// End of an outer step: the outer loop's condition
__global__ void outer_end_kernel(const ProbK* __restrict__ P, int count, ResCtl* ctl,
                                 cudaGraphConditionalHandle h_out) {
  int any = 0;
  for (int p = threadIdx.x; p < count; p += blockDim.x) any |= P[p].rs->open;
  any = __any_sync(0xffffffffu, any);
  if (threadIdx.x == 0) {
    ctl->outer_iters += 1;
    cudaGraphSetConditional(h_out, (any && ctl->outer_iters < ctl->cap_outer) ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct KrylovWork {
  int m = 0;
  int dtype = 0;
  bool flexible = false;
  size_t n = 0;
  void* V = nullptr;
  void* Z = nullptr;
  void* w = nullptr;
  double2* x64 = nullptr;
  double2* r64 = nullptr;
  double2* y64 = nullptr;
  double2* H = nullptr;
  double2* hcol = nullptr;
  double2* h2 = nullptr;
  double2* g = nullptr;
  double2* ysol = nullptr;
  double* cs = nullptr;
  double2* sn = nullptr;
  double2* partial = nullptr;
  double2* Q = nullptr;     // rotation product (cooperative step)
  void* rin = nullptr;      // inner residual (mixed mode)
  void* d = nullptr;        // inner correction (mixed mode)
};

static void free_work(KrylovWork* k) {
  cudaFree(k->V); cudaFree(k->Z); cudaFree(k->w); cudaFree(k->x64); cudaFree(k->r64); cudaFree(k->y64);
  cudaFree(k->H); cudaFree(k->hcol); cudaFree(k->h2); cudaFree(k->g); cudaFree(k->ysol); cudaFree(k->cs);
  cudaFree(k->sn); cudaFree(k->partial); cudaFree(k->Q); cudaFree(k->rin); cudaFree(k->d);
  *k = KrylovWork();
}

static vie_status alloc_work(KrylovWork* k, size_t n, int m, int dtype, bool flexible) {
  const size_t es = dtype == VIE_C64 ? sizeof(float2) : sizeof(double2);
  k->m = m; k->dtype = dtype; k->flexible = flexible; k->n = n;
  struct { void** p; size_t sz; } a[] = {
      {&k->V, (size_t)(m + 1) * n * es}, {&k->w, n * es}, {(void**)&k->x64, n * sizeof(double2)},
      {(void**)&k->r64, n * sizeof(double2)}, {(void**)&k->y64, n * sizeof(double2)},
      {(void**)&k->H, (size_t)(m + 1) * m * sizeof(double2)}, {(void**)&k->hcol, (m + 1) * sizeof(double2)},
      {(void**)&k->h2, (m + 1) * sizeof(double2)}, {(void**)&k->g, (m + 1) * sizeof(double2)},
      {(void**)&k->ysol, (m + 1) * sizeof(double2)}, {(void**)&k->cs, (m + 1) * sizeof(double)},
      {(void**)&k->sn, (m + 1) * sizeof(double2)},
      {(void**)&k->partial, (size_t)(m + 2) * kDotBlocks * sizeof(double2)},
      {(void**)&k->Q, (size_t)(m + 1) * (m + 1) * sizeof(double2)},
      {&k->rin, n * es}, {&k->d, n * es}};
  for (auto& e : a) {
    cudaError_t err = cudaMalloc(e.p, e.sz);
    if (err != cudaSuccess) {
      set_error("solver workspace cudaMalloc(%zu): %s", e.sz, cudaGetErrorString(err));
      free_work(k);
      return VIE_ERR_OOM;
    }
  }
  if (flexible) {
    cudaError_t err = cudaMalloc(&k->Z, (size_t)m * n * es);
    if (err != cudaSuccess) { set_error("solver workspace Z: %s", cudaGetErrorString(err)); free_work(k); return VIE_ERR_OOM; }
  }
  return VIE_OK;
}

void free_krylov(vie_plan* p) {
  if (p && p->krylov) {
    KrylovWork* k = (KrylovWork*)p->krylov;
    free_work(k);
    delete k;
    p->krylov = nullptr;
  }
}

static vie_status ensure_work(vie_plan* p, int m, int dtype, bool flexible, KrylovWork** out, int comps) {
  const size_t n = (size_t)comps * p->n[0] * p->n[1] * p->n[2];
  KrylovWork* k = (KrylovWork*)p->krylov;
  if (k && k->m == m && k->dtype == dtype && k->flexible == flexible && k->n == n) {
    *out = k;
    return VIE_OK;
  }
  free_krylov(p);
  k = new KrylovWork();
  vie_status st = alloc_work(k, n, m, dtype, flexible);
  if (st != VIE_OK) { delete k; return st; }
  p->krylov = k;
  *out = k;
  return VIE_OK;
}

static unsigned grid_for(size_t n) {
  const size_t b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < (size_t)152 * 8 ? b : (size_t)152 * 8);
}

// Per-call state of a (batched) solve.
struct BatchCall {
  std::vector<vie_plan*> plans;
  std::vector<ProbK> host;          // one record per problem
  ProbK* table = nullptr;           // device records of the current list
  SolveStatus* st = nullptr;        // device, one per problem
  SolveStatus* st_host = nullptr;   // pinned mirror
  double2* partial_host = nullptr;  // pinned, kDotBlocks per problem
  std::vector<char> pc_on;          // preconditioner still in use, per problem
  bool jm = false;                  // JM-VIE problems (6N unknowns)
  bool last_cycle_graph = false;    // the last cycle ran as a graph launch
  unsigned* bar = nullptr;          // grid barrier of the cooperative step (arrivals, generation, abort)
  unsigned* bar_host = nullptr;     // pinned copy of the abort word
  int coop_blocks = 0;              // blocks of the cooperative step (0: separate kernels)
  bool resident = false;            // the whole solve runs as one graph launch
  ResState* rs = nullptr;           // device, one per problem (resident solve)
  ResCtl* ctl = nullptr;            // device (resident solve)
  ~BatchCall() {
    cudaFree(rs);
    cudaFree(ctl);
    cudaFree(table);
    cudaFree(st);
    cudaFree(bar);
    cudaFreeHost(st_host);
    cudaFreeHost(partial_host);
    cudaFreeHost(bar_host);
  }
};

// Blocks of the cooperative Gram-Schmidt step for inner type V: one per SM
// at most as many as fit resident, capped at kDotBlocks (the partial-sum
// stride); 0 where cooperative launch is not available.
template <typename V>
static int coop_blocks_for(int m) {
  int dev = 0, coop = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t dyn = (size_t)(m + 1) * sizeof(typename Acc<V>::T) + 16 + (size_t)(2 * m + 2) * sizeof(double2) +
                     (size_t)m * sizeof(double);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, arnoldi_coop_kernel<V>, coop_threads<V>(), dyn) !=
                   cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = sms * (per > 1 ? 1 : per);
  return nb > kDotBlocks ? kDotBlocks : nb;
}

static vie_status upload_list(BatchCall& c, const std::vector<int>& list, cudaStream_t s) {
  std::vector<ProbK> t(list.size());
  for (size_t i = 0; i < list.size(); ++i) t[i] = c.host[list[i]];
  VIE_CUDA_TRY(cudaMemcpyAsync(c.table, t.data(), t.size() * sizeof(ProbK), cudaMemcpyHostToDevice, s));
  // the host vector dies at return: make the copy complete first
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  return VIE_OK;
}

// Operator on z_j (inner type) or on x (complex128, outer) for every problem
// of `list`, grouped by shape.
enum { APPLY_Z = 0, APPLY_X = 1, APPLY_D = 2 };

// Operator on z_j (inner type, -> w), on x (complex128, -> y64) or on the
// last correction d (inner type, -> w) for every problem of `list`, grouped
// by shape.
static vie_status apply_list(BatchCall& c, const std::vector<int>& list, int dtype, int which, int j, bool flexible,
                             cudaStream_t s) {
  const bool outer = which == APPLY_X;
  std::vector<int> used(list.size(), 0);
  const size_t es = dtype == VIE_C64 ? sizeof(float2) : sizeof(double2);
  if (c.jm) {
    // one JM-VIE operator per problem (no grouping)
    for (int i : list) {
      const ProbK& q = c.host[i];
      const void* xin;
      void* yout;
      if (outer) {
        xin = q.x64;
        yout = q.y64;
      } else if (which == APPLY_D) {
        xin = q.d;
        yout = q.w;
      } else {
        xin = (const char*)(flexible ? q.Z : q.V) + (size_t)j * q.n * es;
        yout = q.w;
      }
      vie_status st = jm_matvec_impl(c.plans[i], xin, yout, outer ? VIE_C128 : dtype, MODE_OPERATOR, s);
      if (st != VIE_OK) return st;
    }
    return VIE_OK;
  }
  for (size_t i = 0; i < list.size(); ++i) {
    if (used[i]) continue;
    std::vector<vie_plan*> gp;
    std::vector<const void*> gx;
    std::vector<void*> gy;
    std::vector<const int*> gl;       // per plan the device flag that skips it when 0
    const vie_plan* a = c.plans[list[i]];
    for (size_t k = i; k < list.size(); ++k) {
      if (used[k]) continue;
      const vie_plan* b = c.plans[list[k]];
      if (a->n[0] == b->n[0] && a->n[1] == b->n[1] && a->n[2] == b->n[2] && a->m[0] == b->m[0] &&
          a->m[1] == b->m[1] && a->m[2] == b->m[2]) {
        const ProbK& q = c.host[list[k]];
        const int pi = list[k];
        used[k] = 1;
        gp.push_back(c.plans[list[k]]);
        if (outer) {
          gx.push_back(q.x64);
          gy.push_back(q.y64);
          gl.push_back(c.resident ? &c.rs[pi].open : nullptr);
        } else if (which == APPLY_D) {
          gx.push_back(q.d);
          gy.push_back(q.w);
          gl.push_back(c.resident ? &c.rs[pi].inner : nullptr);
        } else {
          // an Arnoldi step: problems that stopped in this cycle are skipped
          const char* zb = (const char*)(flexible ? q.Z : q.V);
          gx.push_back(zb + (size_t)j * q.n * es);
          gy.push_back(q.w);
          gl.push_back(&c.st[pi].active);
        }
      }
    }
    vie_status st = matvec_group(gp.data(), (int)gp.size(), gx.data(), gy.data(), outer ? VIE_C128 : dtype,
                                 MODE_OPERATOR, s, gl.data());
    if (st != VIE_OK) return st;
  }
  return VIE_OK;
}

static vie_status read_status(BatchCall& c, cudaStream_t s) {
  VIE_CUDA_TRY(cudaMemcpyAsync(c.st_host, c.st, c.plans.size() * sizeof(SolveStatus), cudaMemcpyDeviceToHost, s));
  if (c.bar) VIE_CUDA_TRY(cudaMemcpyAsync(c.bar_host, c.bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (c.bar && *c.bar_host) {
    set_error("a grid barrier of the Gram-Schmidt step timed out");
    return VIE_ERR_TIMEOUT;
  }
  return VIE_OK;
}

// One Arnoldi step j for the problems of `list`: preconditioner (flexible),
// operator, Gram-Schmidt with the device-side second-pass decision, the FP64
// Givens step and the next basis vector.  Problems whose status is inactive
// return at once from every Krylov kernel.
// `list` is the table the kernels index (all problems of the cycle), `live`
// the problems whose preconditioner and operator are applied.
template <typename V>
static vie_status enqueue_step(BatchCall& c, const std::vector<int>& list, const std::vector<int>& live, int j, int m,
                               int dtype, bool flexible, vie_precond_fn precond, void* const* precond_ctx,
                               unsigned gx, cudaStream_t s, cudaGraphConditionalHandle next = 0,
                               bool* next_set = nullptr) {
  if (next_set) *next_set = false;
  const unsigned P = (unsigned)list.size();
  if (flexible) {
    for (int i : live) {
      const ProbK& q = c.host[i];
      const char* vj = (const char*)q.V + (size_t)j * q.n * sizeof(V);
      char* zj = (char*)q.Z + (size_t)j * q.n * sizeof(V);
      if (c.pc_on[i]) {
        vie_status ps = precond(precond_ctx[i], dtype, vj, zj, s);
        if (ps != VIE_OK) return ps;
      } else {
        VIE_CUDA_TRY(cudaMemcpyAsync(zj, vj, q.n * sizeof(V), cudaMemcpyDeviceToDevice, s));
      }
    }
  }
  vie_status ms = apply_list(c, live, dtype, APPLY_Z, j, flexible, s);
  if (ms != VIE_OK) return ms;
  const int nv = j + 1;
  if (c.coop_blocks > 0 && P <= (unsigned)kCoopMaxProblems) {
    // the whole Gram-Schmidt step, ||w||, v_{j+1} and the Givens step in one
    // cooperative launch
    const size_t dyn = ((nv * sizeof(typename Acc<V>::T) + 15) / 16) * 16 + (size_t)(2 * j + 2) * sizeof(double2) +
                       (size_t)j * sizeof(double);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c.coop_blocks);
    cfg.blockDim = dim3(coop_threads<V>());
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int set_next = next_set ? 1 : 0;
    VIE_CUDA_TRY(cudaLaunchKernelEx(&cfg, arnoldi_coop_kernel<V>, (const ProbK*)c.table, (int)P, nv, m + 1, c.bar,
                                    next, set_next));
    if (next_set) *next_set = true;
    return VIE_OK;
  }
  // h1 = V^H w, w -= V h1 (+ norm); if needed h2 = V^H w, w -= V h2 (+ norm); column h1 + h2
  const dim3 gdots(kDotBlocks, (unsigned)((nv + kGroup - 1) / kGroup), P);
  const size_t hs_bytes = nv * sizeof(typename Acc<V>::T);
  dots_kernel<V><<<gdots, kThreads, 0, s>>>(c.table, nv, 0);
  reduce_partials_kernel<<<dim3(nv, P), kThreads, 0, s>>>(c.table, kDotBlocks, 0);
  update_kernel<V><<<dim3(gx, P), kThreads, hs_bytes, s>>>(c.table, nv, 0);
  reorth_decide_kernel<<<P, kThreads, 0, s>>>(c.table, (int)gx, nv);
  dots_kernel<V><<<gdots, kThreads, 0, s>>>(c.table, nv, 1);
  reduce_partials_kernel<<<dim3(nv, P), kThreads, 0, s>>>(c.table, kDotBlocks, 1);
  update_kernel<V><<<dim3(gx, P), kThreads, hs_bytes, s>>>(c.table, nv, 1);
  arnoldi_step_kernel<<<P, kThreads, 0, s>>>(c.table, (int)gx, m + 1, j);
  next_vector_kernel<V><<<dim3(gx, P), kThreads, 0, s>>>(c.table, j);
  VIE_LAUNCH_CHECK();
  return VIE_OK;
}

// Condition of the next step's graph node: 1 while any problem of the list
// is still active.
__global__ void next_step_condition_kernel(const ProbK* __restrict__ P, int count, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int i = 0; i < count; ++i) any |= P[i].st->active;
  cudaGraphSetConditional(h, any ? 1u : 0u);
}

// A whole GMRES cycle as one CUDA graph: the start vector, then one
// conditional (IF) node per Arnoldi step whose body ends by setting the next
// step's condition from the problems' device status, then the back
// substitution and the update of x.  Launched once per cycle, it runs every
// step on the device with no host round trip; the steps after the last
// active problem stopped are skipped by the device.  The instantiated graph
// is kept while the list of problems, the preconditioner switches and the
// step count stay the same (the records' table is one device buffer).
struct CycleGraph {
  std::vector<int> list;
  std::vector<char> pc;
  int jmax = 0, m = 0, dtype = 0;
  bool flexible = false;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = nullptr;
  bool broken = false;         // capture or instantiation failed once: use the host loop
  ~CycleGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  }
};

template <typename V>
static vie_status build_cycle_graph(BatchCall& c, CycleGraph& G, const std::vector<int>& list, int m, int jmax,
                                    int dtype, bool flexible, vie_precond_fn precond, void* const* precond_ctx,
                                    unsigned gx) {
  if (G.exec) { cudaGraphExecDestroy(G.exec); G.exec = nullptr; }
  if (G.graph) { cudaGraphDestroy(G.graph); G.graph = nullptr; }
  if (!G.cap) VIE_CUDA_TRY(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
  const unsigned P = (unsigned)list.size();
  VIE_CUDA_TRY(cudaGraphCreate(&G.graph, 0));
  // handles: [0] start (always), [1 + j] step j (step 0 always, later steps
  // set by the step before), [jmax + 1] finish (always)
  std::vector<cudaGraphConditionalHandle> h(jmax + 2);
  for (int k = 0; k < jmax + 2; ++k) {
    const unsigned def = (k == 0 || k == 1 || k == jmax + 1) ? 1u : 0u;
    VIE_CUDA_TRY(cudaGraphConditionalHandleCreate(&h[k], G.graph, def, cudaGraphCondAssignDefault));
  }
  cudaGraphNode_t prev = nullptr;
  for (int k = 0; k < jmax + 2; ++k) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h[k];
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    VIE_CUDA_TRY(cudaGraphAddNode(&node, G.graph, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    VIE_CUDA_TRY(cudaStreamBeginCaptureToGraph(G.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    vie_status st = VIE_OK;
    if (k == 0) {
      start_vector_kernel<V><<<dim3(gx, P), kThreads, 0, G.cap>>>(c.table);
    } else if (k <= jmax) {
      bool set = false;
      st = enqueue_step<V>(c, list, list, k - 1, m, dtype, flexible, precond, precond_ctx, gx, G.cap,
                           k < jmax ? h[k + 1] : 0, k < jmax ? &set : nullptr);
      if (st == VIE_OK && k < jmax && !set)
        next_step_condition_kernel<<<1, 32, 0, G.cap>>>(c.table, (int)P, h[k + 1]);
    } else {
      backsolve_kernel<<<P, kThreads, 0, G.cap>>>(c.table, m + 1);
      update_x_kernel<V><<<dim3(gx, P), kThreads, (size_t)m * sizeof(typename Acc<V>::T), G.cap>>>(c.table);
    }
    cudaGraph_t out = body;
    cudaError_t e = cudaStreamEndCapture(G.cap, &out);
    if (st != VIE_OK) return st;
    if (e != cudaSuccess) {
      set_error("capture of a GMRES step: %s", cudaGetErrorString(e));
      return VIE_ERR_CUDA;
    }
    prev = node;
  }
  VIE_CUDA_TRY(cudaGraphInstantiate(&G.exec, G.graph, 0));
  G.list = list;
  G.pc.clear();
  for (int i : list) G.pc.push_back(c.pc_on[i]);
  G.jmax = jmax;
  G.m = m;
  G.dtype = dtype;
  G.flexible = flexible;
  return VIE_OK;
}

// One GMRES cycle of at most m steps for the problems of `list` (whose
// records are on the device and whose status was just initialised): as one
// graph launch (above), or, if the graph cannot be built, from the host with
// a status read every check_every steps.
template <typename V>
static vie_status run_cycle(BatchCall& c, CycleGraph& G, const std::vector<int>& list, int m, int dtype,
                            int max_steps, int check_every, bool flexible, vie_precond_fn precond,
                            void* const* precond_ctx, cudaStream_t s) {
  const unsigned P = (unsigned)list.size();
  size_t nmax = 0;
  for (int i : list) nmax = c.host[i].n > nmax ? c.host[i].n : nmax;
  const unsigned gx = grid_for(nmax);
  const int jmax = max_steps < m ? max_steps : m;
  if (!G.broken) {
    std::vector<char> pc;
    for (int i : list) pc.push_back(c.pc_on[i]);
    const bool same = G.exec && G.list == list && G.pc == pc && G.jmax == jmax && G.m == m && G.dtype == dtype &&
                      G.flexible == flexible;
    vie_status st = VIE_OK;
    if (!same) {
      st = build_cycle_graph<V>(c, G, list, m, jmax, dtype, flexible, precond, precond_ctx, gx);
      if (st != VIE_OK) {
        // conditional graph nodes unavailable here: fall back to the host loop
        G.broken = true;
        cudaGetLastError();
        clear_error();
      }
    }
    if (!G.broken) {
      VIE_CUDA_TRY(cudaGraphLaunch(G.exec, s));
      c.last_cycle_graph = true;
      return read_status(c, s);
    }
  }
  c.last_cycle_graph = false;
  start_vector_kernel<V><<<dim3(gx, P), kThreads, 0, s>>>(c.table);
  VIE_LAUNCH_CHECK();
  std::vector<int> live = list;       // problems still iterating in this cycle
  for (int j = 0; j < jmax && !live.empty(); ++j) {
    vie_status st = enqueue_step<V>(c, list, live, j, m, dtype, flexible, precond, precond_ctx, gx, s);
    if (st != VIE_OK) return st;
    if ((j + 1) % check_every == 0 || j + 1 == jmax) {
      vie_status rs = read_status(c, s);
      if (rs != VIE_OK) return rs;
      std::vector<int> still;
      for (int i : live)
        if (c.st_host[i].active) still.push_back(i);
      live.swap(still);
    }
  }
  backsolve_kernel<<<P, kThreads, 0, s>>>(c.table, m + 1);
  update_x_kernel<V><<<dim3(gx, P), kThreads, (size_t)m * sizeof(typename Acc<V>::T), s>>>(c.table);
  VIE_LAUNCH_CHECK();
  return read_status(c, s);
}

// ---------------------------------------------------------------------------
// Device-resident solve: the whole refinement loop as one graph launch
// ---------------------------------------------------------------------------
// Appends a conditional node (handle h, IF or WHILE) after *prev in g and
// returns its body graph; *prev becomes the new node.
static vie_status add_cond(cudaGraph_t g, cudaGraphNode_t* prev, cudaGraphConditionalHandle h,
                           cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  VIE_CUDA_TRY(cudaGraphAddNode(&node, g, *prev ? prev : nullptr, nullptr, *prev ? 1 : 0, &cp));
  *body = cp.conditional.phGraph_out[0];
  *prev = node;
  return VIE_OK;
}

// Appends a segment of launches, captured from fn(stream), as the body of an
// always-true IF node (so that segments and conditional nodes chain by
// explicit dependencies).
template <typename F>
static vie_status add_segment(cudaGraph_t g, cudaGraphNode_t* prev, cudaStream_t cap, F fn) {
  cudaGraphConditionalHandle h;
  VIE_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraph_t body;
  vie_status st = add_cond(g, prev, h, cudaGraphCondTypeIf, &body);
  if (st != VIE_OK) return st;
  VIE_CUDA_TRY(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  st = fn(cap);
  cudaGraph_t out = body;
  const cudaError_t e = cudaStreamEndCapture(cap, &out);
  if (st != VIE_OK) return st;
  if (e != cudaSuccess) {
    set_error("capture into a solve graph: %s", cudaGetErrorString(e));
    return VIE_ERR_CUDA;
  }
  return VIE_OK;
}

struct ResidentGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphConditionalHandle* steps_dev = nullptr;   // the step handles, for reset_steps_kernel
  ~ResidentGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(steps_dev);
  }
};

// Captures fn(stream) into an existing (conditional body) graph.
template <typename F>
static vie_status capture_into(cudaGraph_t body, cudaStream_t cap, F fn) {
  VIE_CUDA_TRY(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  vie_status st = fn(cap);
  cudaGraph_t out = body;
  const cudaError_t e = cudaStreamEndCapture(cap, &out);
  if (st != VIE_OK) return st;
  if (e != cudaSuccess) {
    set_error("capture into a solve graph: %s", cudaGetErrorString(e));
    return VIE_ERR_CUDA;
  }
  return VIE_OK;
}

// The solve as one graph (plain GMRES or mixed-precision refinement, no
// preconditioner), all problems in c.table with their ResState:
//   WHILE (any problem open, outer steps < cap)
//     A x (complex128, open problems), r = b - A x, outer_decide,
//     [mixed: rin = r in complex64]
//     WHILE (any problem with an inner cycle, rounds < kMaxInnerCycles)
//       init_cycle, reset of the step conditions, start vector
//       IF step 0 .. IF step jmax-1 (each sets the next step's condition)
//       back substitution, x += Z y
//       inner_decide, [mixed: A d and rin -= A d for problems going on]
//     outer_end
template <typename V>
static vie_status build_resident_graph(BatchCall& c, ResidentGraph& R, const std::vector<int>& all, int m,
                                       int jmax, int dtype, bool mixed, double tol, double inner_tol, int max_iters,
                                       int max_outer, unsigned gx) {
  const unsigned P = (unsigned)all.size();
  const int mx = mixed ? 1 : 0;
  VIE_CUDA_TRY(cudaStreamCreateWithFlags(&R.cap, cudaStreamNonBlocking));
  VIE_CUDA_TRY(cudaGraphCreate(&R.graph, 0));
  cudaGraphConditionalHandle h_out, h_in;
  VIE_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_out, R.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNode_t top = nullptr;
  cudaGraph_t B_out, B_in;
  vie_status st = add_cond(R.graph, &top, h_out, cudaGraphCondTypeWhile, &B_out);
  if (st != VIE_OK) return st;
  VIE_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_in, B_out, 0, cudaGraphCondAssignDefault));
  cudaGraphNode_t po = nullptr;
  st = add_segment(B_out, &po, R.cap, [&](cudaStream_t cs) -> vie_status {
    vie_status a = apply_list(c, all, dtype, APPLY_X, 0, false, cs);
    if (a != VIE_OK) return a;
    residual_kernel<<<dim3(kDotBlocks, P), kThreads, 0, cs>>>(c.table);
    outer_decide_kernel<<<P, kThreads, 0, cs>>>(c.table, kDotBlocks, tol, inner_tol, mx, max_iters, max_outer, c.ctl);
    outer_finalize_kernel<<<1, 32, 0, cs>>>(c.table, (int)P, c.ctl, h_in);
    if (mixed) inner_from_outer_kernel<float2><<<dim3(kDotBlocks, P), kThreads, 0, cs>>>(c.table);
    VIE_LAUNCH_CHECK();
    return VIE_OK;
  });
  if (st != VIE_OK) return st;
  st = add_cond(B_out, &po, h_in, cudaGraphCondTypeWhile, &B_in);
  if (st != VIE_OK) return st;
  st = add_segment(B_out, &po, R.cap, [&](cudaStream_t cs) -> vie_status {
    outer_end_kernel<<<1, 32, 0, cs>>>(c.table, (int)P, c.ctl, h_out);
    VIE_LAUNCH_CHECK();
    return VIE_OK;
  });
  if (st != VIE_OK) return st;
  // the inner loop's body: one cycle
  std::vector<cudaGraphConditionalHandle> hs(jmax);
  for (int k = 0; k < jmax; ++k)
    VIE_CUDA_TRY(cudaGraphConditionalHandleCreate(&hs[k], B_in, k == 0 ? 1 : 0, cudaGraphCondAssignDefault));
  VIE_CUDA_TRY(cudaMalloc((void**)&R.steps_dev, jmax * sizeof(cudaGraphConditionalHandle)));
  VIE_CUDA_TRY(cudaMemcpy(R.steps_dev, hs.data(), jmax * sizeof(cudaGraphConditionalHandle), cudaMemcpyHostToDevice));
  cudaGraphNode_t pi = nullptr;
  st = add_segment(B_in, &pi, R.cap, [&](cudaStream_t cs) -> vie_status {
    init_cycle_kernel<<<P, kThreads, 0, cs>>>(c.table, kDotBlocks, m);
    reset_steps_kernel<<<1, 256, 0, cs>>>(R.steps_dev, jmax);
    start_vector_kernel<V><<<dim3(gx, P), kThreads, 0, cs>>>(c.table);
    VIE_LAUNCH_CHECK();
    return VIE_OK;
  });
  if (st != VIE_OK) return st;
  for (int k = 0; k < jmax; ++k) {
    cudaGraph_t body;
    st = add_cond(B_in, &pi, hs[k], cudaGraphCondTypeIf, &body);
    if (st != VIE_OK) return st;
    st = capture_into(body, R.cap, [&](cudaStream_t cs) -> vie_status {
      bool set = false;
      const bool last = k + 1 >= jmax;
      vie_status e = enqueue_step<V>(c, all, all, k, m, dtype, false, nullptr, nullptr, gx, cs,
                                     last ? 0 : hs[k + 1], last ? nullptr : &set);
      if (e != VIE_OK) return e;
      if (!last && !set) next_step_condition_kernel<<<1, 32, 0, cs>>>(c.table, (int)P, hs[k + 1]);
      VIE_LAUNCH_CHECK();
      return VIE_OK;
    });
    if (st != VIE_OK) return st;
  }
  st = add_segment(B_in, &pi, R.cap, [&](cudaStream_t cs) -> vie_status {
    backsolve_kernel<<<P, kThreads, 0, cs>>>(c.table, m + 1);
    update_x_kernel<V><<<dim3(gx, P), kThreads, (size_t)m * sizeof(typename Acc<V>::T), cs>>>(c.table);
    inner_decide_kernel<<<1, 32, 0, cs>>>(c.table, (int)P, mx, max_iters, c.ctl, h_in);
    VIE_LAUNCH_CHECK();
    if (mixed) {
      vie_status a = apply_list(c, all, dtype, APPLY_D, 0, false, cs);
      if (a != VIE_OK) return a;
      inner_residual_kernel<float2><<<dim3(kDotBlocks, P), kThreads, 0, cs>>>(c.table);
      VIE_LAUNCH_CHECK();
    }
    return VIE_OK;
  });
  if (st != VIE_OK) return st;
  VIE_CUDA_TRY(cudaGraphInstantiate(&R.exec, R.graph, 0));
  return VIE_OK;
}

// The solve as one graph launch (build_resident_graph).  *used = false when
// the graph cannot be built here; the caller then runs the host loop.
template <typename V>
static vie_status solve_resident(BatchCall& c, int count, int m, int dtype, bool mixed, double tol,
                                 double inner_tol, int max_iters, int max_outer, double timeout,
                                 double2* const* x, vie_solve_info* infos, cudaStream_t s, bool* used) {
  *used = false;
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) all[i] = i;
  VIE_CUDA_TRY(cudaMalloc((void**)&c.rs, count * sizeof(ResState)));
  VIE_CUDA_TRY(cudaMalloc((void**)&c.ctl, sizeof(ResCtl)));
  std::vector<ResState> rh(count);
  memset(rh.data(), 0, count * sizeof(ResState));
  for (int i = 0; i < count; ++i) {
    rh[i].open = c.host[i].bnorm != 0.0 ? 1 : 0;
    rh[i].converged = c.host[i].bnorm == 0.0 ? 1 : 0;
    c.host[i].rs = c.rs + i;
    c.host[i].from_inner = mixed ? 1 : 0;
  }
  ResCtl ch;
  memset(&ch, 0, sizeof(ch));
  ch.limit_ns = (unsigned long long)(timeout * 1e9);
  ch.cap_outer = max_outer + 2;
  VIE_CUDA_TRY(cudaMemcpyAsync(c.rs, rh.data(), count * sizeof(ResState), cudaMemcpyHostToDevice, s));
  VIE_CUDA_TRY(cudaMemcpyAsync(c.ctl, &ch, sizeof(ResCtl), cudaMemcpyHostToDevice, s));
  c.resident = true;
  vie_status st = upload_list(c, all, s);   // synchronises: the host copies above have landed
  if (st != VIE_OK) return st;
  size_t nmax = 0;
  for (int i = 0; i < count; ++i) nmax = c.host[i].n > nmax ? c.host[i].n : nmax;
  const unsigned gx = grid_for(nmax);
  const int jmax = max_iters < m ? max_iters : m;
  ResidentGraph R;
  st = build_resident_graph<V>(c, R, all, m, jmax, dtype, mixed, tol, inner_tol, max_iters, max_outer, gx);
  if (st != VIE_OK) {
    // conditional graph nodes unavailable here: the host loop takes over
    cudaGetLastError();
    clear_error();
    c.resident = false;
    for (int i = 0; i < count; ++i) c.host[i].rs = nullptr;
    return VIE_OK;
  }
  *used = true;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  VIE_CUDA_TRY(cudaGraphLaunch(R.exec, s));
  cudaEventRecord(e1, s);
  for (int i = 0; i < count; ++i)
    VIE_CUDA_TRY(cudaMemcpyAsync(x[i], c.host[i].x64, c.host[i].n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  st = read_status(c, s);   // also reports a grid barrier that gave up
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != VIE_OK) return st;
  VIE_CUDA_TRY(cudaMemcpy(rh.data(), c.rs, count * sizeof(ResState), cudaMemcpyDeviceToHost));
  vie_status worst = VIE_OK;
  bool timed_out = false;
  for (int i = 0; i < count; ++i) {
    const ResState& r = rh[i];
    vie_solve_info& inf = infos[i];
    inf.iterations = r.iters;
    inf.outer = r.outers;
    inf.residual = c.host[i].bnorm != 0.0 ? r.rel : 0.0;
    inf.converged = r.converged;
    inf.matvecs64 += r.matvecs64;
    inf.matvecs32 += r.matvecs32;
    inf.graph_cycles = r.graph_cycles;
    inf.reorth_steps = r.reorth_steps;
    inf.history_len = r.hist_len;
    for (int k = 0; k < r.hist_len && k < 64; ++k) inf.history[k] = r.history[k];
    inf.time_ms = ms;
    vie_status res = (vie_status)r.result;
    if (!r.converged && res == VIE_OK) res = VIE_ERR_NOT_CONVERGED;   // the loops' own caps
    if (res == VIE_ERR_TIMEOUT) timed_out = true;
    if (worst == VIE_OK && res != VIE_OK) worst = res;
  }
  if (timed_out) set_error("solve exceeded %.1f s", timeout);
  else if (worst == VIE_ERR_NOT_CONVERGED) set_error("not converged: a problem stopped above the tolerance (see its info)");
  return worst;
}

// Solve `count` problems; b[i], x[i] complex128 device vectors of plan i.
vie_status solve_batch_impl(vie_plan* const* plans, int count, const double2* const* b, double2* const* x, double tol,
                            const vie_solve_opts* o, vie_solve_info* infos, vie_precond_fn precond,
                            void* const* precond_ctx, cudaStream_t s, int jm) {
  const auto t0 = std::chrono::steady_clock::now();
  const int mode = o->mode;
  const int m = o->restart > 0 ? o->restart : 100;
  if (m > kMaxRestart) { set_error("restart must be <= %d", kMaxRestart); return VIE_ERR_INVALID; }
  const int max_iters = o->max_iters > 0 ? o->max_iters : 5000;
  const int max_outer = o->max_outer > 0 ? o->max_outer : 200;
  const double inner_tol = o->inner_tol > 0 ? o->inner_tol : 1e-4;
  const int check_every = o->check_every > 0 ? o->check_every : 4;
  const double timeout = o->timeout_s > 0 ? o->timeout_s : 600.0;
  const int dtype = (mode == VIE_SOLVE_MIXED) ? VIE_C64 : VIE_C128;
  const bool flexible = precond != nullptr;
  BatchCall c;
  CycleGraph graph;
  c.jm = jm != 0;
  c.plans.assign(plans, plans + count);
  c.host.resize(count);
  c.pc_on.assign(count, flexible ? 1 : 0);
  VIE_CUDA_TRY(cudaMalloc((void**)&c.table, count * sizeof(ProbK)));
  VIE_CUDA_TRY(cudaMalloc((void**)&c.st, count * sizeof(SolveStatus)));
  VIE_CUDA_TRY(cudaMallocHost((void**)&c.st_host, count * sizeof(SolveStatus)));
  VIE_CUDA_TRY(cudaMallocHost((void**)&c.partial_host, (size_t)count * kDotBlocks * sizeof(double2)));
  VIE_CUDA_TRY(cudaMemsetAsync(c.st, 0, count * sizeof(SolveStatus), s));
  VIE_CUDA_TRY(cudaMalloc((void**)&c.bar, 4 * sizeof(unsigned)));
  VIE_CUDA_TRY(cudaMallocHost((void**)&c.bar_host, sizeof(unsigned)));
  VIE_CUDA_TRY(cudaMemsetAsync(c.bar, 0, 4 * sizeof(unsigned), s));
  c.coop_blocks = (count <= kCoopMaxProblems)
                      ? (dtype == VIE_C64 ? coop_blocks_for<float2>(m) : coop_blocks_for<double2>(m))
                      : 0;
  for (int i = 0; i < count; ++i) {
    KrylovWork* k = nullptr;
    vie_status st = ensure_work(plans[i], m, dtype, flexible, &k, jm ? 6 : 3);
    if (st != VIE_OK) return st;
    ProbK& q = c.host[i];
    memset(&q, 0, sizeof(q));
    q.V = k->V; q.Z = flexible ? k->Z : k->V; q.w = k->w; q.n = k->n; q.b = b[i];
    q.x64 = k->x64; q.r64 = k->r64; q.y64 = k->y64; q.H = k->H; q.hcol = k->hcol; q.h2 = k->h2; q.g = k->g;
    q.ysol = k->ysol; q.cs = k->cs; q.sn = k->sn; q.partial = k->partial; q.Q = k->Q; q.st = c.st + i;
    q.rin = k->rin; q.d = mode == VIE_SOLVE_MIXED ? k->d : nullptr; q.from_inner = 0;
    memset(&infos[i], 0, sizeof(vie_solve_info));
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) all[i] = i;
  // ||b|| of every problem
  vie_status st = upload_list(c, all, s);
  if (st != VIE_OK) return st;
  norm2_b_kernel<<<dim3(kDotBlocks, count), kThreads, 0, s>>>(c.table);
  VIE_LAUNCH_CHECK();
  for (int i = 0; i < count; ++i)
    VIE_CUDA_TRY(cudaMemcpyAsync(c.partial_host + (size_t)i * kDotBlocks, c.host[i].partial,
                                 kDotBlocks * sizeof(double2), cudaMemcpyDeviceToHost, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int> list;
  std::vector<int> iters(count, 0), outers(count, 0);
  std::vector<double> rel(count, 0.0), prev_rel(count, 0.0);
  std::vector<vie_status> result(count, VIE_OK);
  std::vector<int> trial(count, 0);         // preconditioner judging: 0 not yet, 1 plain cycle running, 2 done
  std::vector<double> pc_rate(count, 0.0);  // log residual reduction per step of the preconditioned cycle
  for (int i = 0; i < count; ++i) {
    double t = 0.0;
    for (int k = 0; k < kDotBlocks; ++k) t += c.partial_host[(size_t)i * kDotBlocks + k].x;
    c.host[i].bnorm = sqrt(t);
    if (!isfinite(c.host[i].bnorm)) { set_error("right-hand side %d is not finite", i); return VIE_ERR_NONFINITE; }
    if (o->x0_given && c.host[i].bnorm != 0.0) {
      VIE_CUDA_TRY(cudaMemcpyAsync(c.host[i].x64, x[i], c.host[i].n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    } else {
      VIE_CUDA_TRY(cudaMemsetAsync(c.host[i].x64, 0, c.host[i].n * sizeof(double2), s));
    }
    if (c.host[i].bnorm == 0.0) {
      infos[i].converged = 1;
    } else {
      list.push_back(i);
    }
  }
  // without a preconditioner, on request: the whole loop as one graph launch
  if (o->resident && !flexible && !jm && !list.empty()) {
    bool used = false;
    vie_status rs_st = dtype == VIE_C64
                           ? solve_resident<float2>(c, count, m, dtype, mode == VIE_SOLVE_MIXED, tol, inner_tol,
                                                    max_iters, max_outer, timeout, x, infos, s, &used)
                           : solve_resident<double2>(c, count, m, dtype, mode == VIE_SOLVE_MIXED, tol, inner_tol,
                                                     max_iters, max_outer, timeout, x, infos, s, &used);
    if (used || rs_st != VIE_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rs_st;
    }
  }
  st = VIE_OK;
  while (!list.empty()) {
    // true residual r = b - A64 x of the open problems
    st = upload_list(c, list, s);
    if (st != VIE_OK) break;
    st = apply_list(c, list, dtype, APPLY_X, 0, false, s);
    if (st != VIE_OK) break;
    residual_kernel<<<dim3(kDotBlocks, (unsigned)list.size()), kThreads, 0, s>>>(c.table);
    init_cycle_kernel<<<(unsigned)list.size(), kThreads, 0, s>>>(c.table, kDotBlocks, m);
    VIE_LAUNCH_CHECK();
    st = read_status(c, s);
    if (st != VIE_OK) break;
    std::vector<int> open;
    for (int i : list) {
      infos[i].matvecs64++;
      const double rn = c.st_host[i].beta;
      rel[i] = rn / c.host[i].bnorm;
      if (outers[i] < 64) infos[i].history[outers[i]] = rel[i];
      infos[i].history_len = outers[i] + 1 < 64 ? outers[i] + 1 : 64;
      if (!isfinite(rn)) { result[i] = VIE_ERR_NONFINITE; continue; }
      if (rn <= tol * c.host[i].bnorm) { infos[i].converged = 1; continue; }
      // the true residual judges the preconditioner across refinement steps
      if (c.pc_on[i] && outers[i] > 0 && rel[i] > 0.9 * prev_rel[i]) {
        c.pc_on[i] = 0;
        infos[i].fallback = 1;
        trial[i] = 2;
      }
      prev_rel[i] = rel[i];
      if (iters[i] >= max_iters || outers[i] >= max_outer) { result[i] = VIE_ERR_NOT_CONVERGED; continue; }
      // plain mode goes for tol ||b||; mixed asks the complex64 cycle for a
      // reduction inner_tol, never below half the outer target
      double target = tol * c.host[i].bnorm;
      if (mode == VIE_SOLVE_MIXED) target = fmax(inner_tol * rn, 0.5 * tol * c.host[i].bnorm);
      c.host[i].target = target;
      open.push_back(i);
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!open.empty() && secs > timeout) {
      for (int i : open) result[i] = VIE_ERR_TIMEOUT;
      set_error("solve exceeded %.1f s", timeout);
      open.clear();
    }
    list.swap(open);
    if (list.empty()) break;
    // One refinement step.  Plain mode: one complex128 cycle from r.  Mixed
    // mode: complex64 cycles towards the step's target, each restarted from
    // the complex64 residual r <- r - A d (d = the cycle's correction), so the
    // complex128 operator runs once per step instead of once per cycle.
    std::vector<int> inner = list, next;
    for (int i : list) c.host[i].from_inner = (mode == VIE_SOLVE_MIXED) ? 1 : 0;
    st = upload_list(c, inner, s);
    if (st != VIE_OK) break;
    if (mode == VIE_SOLVE_MIXED) {
      inner_from_outer_kernel<float2><<<dim3(kDotBlocks, (unsigned)inner.size()), kThreads, 0, s>>>(c.table);
      VIE_LAUNCH_CHECK();
    }
    for (int round = 0; !inner.empty(); ++round) {
      init_cycle_kernel<<<(unsigned)inner.size(), kThreads, 0, s>>>(c.table, kDotBlocks, m);
      VIE_LAUNCH_CHECK();
      int steps_left = max_iters;
      for (int i : inner) steps_left = (max_iters - iters[i]) < steps_left ? (max_iters - iters[i]) : steps_left;
      if (dtype == VIE_C64)
        st = run_cycle<float2>(c, graph, inner, m, dtype, steps_left, check_every, flexible, precond, precond_ctx,
                               s);
      else
        st = run_cycle<double2>(c, graph, inner, m, dtype, steps_left, check_every, flexible, precond,
                                precond_ctx, s);
      if (st != VIE_OK) break;
      std::vector<int> again;
      for (int i : inner) {
        const int steps = c.st_host[i].j;
        infos[i].graph_cycles += c.last_cycle_graph ? 1 : 0;
        infos[i].reorth_steps += c.st_host[i].reorth_count;
        iters[i] += steps;
        if (dtype == VIE_C64) infos[i].matvecs32 += steps; else infos[i].matvecs64 += steps;
        if (steps == 0) {
          result[i] = VIE_ERR_NOT_CONVERGED;
          set_error("Krylov cycle made no progress (breakdown at the first step) for problem %d", i);
          continue;
        }
        // The true residual judges the preconditioner against plain GMRES.  A
        // preconditioned cycle that cut the residual by less than 10 %, or a
        // non-finite network output, switches this problem to the identity.
        // For a learned network (whose quality nothing guarantees) the first
        // preconditioned cycle that ends without reaching its target is
        // followed by one plain cycle; the network is kept only if its cycle
        // reduced the residual faster per step.
        const SolveStatus& sh = c.st_host[i];
        const double rate = (steps > 0 && sh.resid > 0.0 && sh.beta > 0.0) ? log(sh.beta / sh.resid) / steps : 0.0;
        if (trial[i] == 1) {
          trial[i] = 2;
          if (rate >= pc_rate[i]) infos[i].fallback = 1;   // plain was as fast: stay plain
          else c.pc_on[i] = 1;
        } else if (c.pc_on[i] && !sh.converged) {
          const bool stalled = sh.resid > 0.9 * sh.beta;
          const bool broken = precond_fallback_flag(c.plans[i], 1) != 0;
          if (stalled || broken) {
            c.pc_on[i] = 0;
            infos[i].fallback = 1;
            trial[i] = 2;
          } else if (trial[i] == 0 && !sh.breakdown && precond_is_learned(c.plans[i])) {
            pc_rate[i] = rate;
            trial[i] = 1;
            c.pc_on[i] = 0;
          }
        }
        const bool more = mode == VIE_SOLVE_MIXED && !c.st_host[i].converged && !c.st_host[i].breakdown &&
                          round + 1 < kMaxInnerCycles && iters[i] < max_iters;
        if (more) again.push_back(i); else next.push_back(i);
      }
      if (again.empty()) break;
      st = upload_list(c, again, s);
      if (st != VIE_OK) break;
      st = apply_list(c, again, dtype, APPLY_D, 0, false, s);
      if (st != VIE_OK) break;
      inner_residual_kernel<float2><<<dim3(kDotBlocks, (unsigned)again.size()), kThreads, 0, s>>>(c.table);
      VIE_LAUNCH_CHECK();
      for (int i : again) infos[i].matvecs32++;
      inner.swap(again);
    }
    if (st != VIE_OK) break;
    for (int i : next) outers[i]++;
    list.swap(next);
  }
  cudaEventRecord(e1, s);
  for (int i = 0; i < count; ++i)
    VIE_CUDA_TRY(cudaMemcpyAsync(x[i], c.host[i].x64, c.host[i].n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  vie_status worst = st;
  for (int i = 0; i < count; ++i) {
    // a network whose outputs had to be replaced (non-finite) counts as
    // dropped even when the solve converged before the per-cycle check
    if (flexible && precond_fallback_flag(c.plans[i], 1)) infos[i].fallback = 1;
    infos[i].iterations = iters[i];
    infos[i].outer = outers[i];
    infos[i].residual = rel[i];
    infos[i].time_ms = ms;
    if (worst == VIE_OK && result[i] != VIE_OK) worst = result[i];
  }
  if (worst == VIE_ERR_NOT_CONVERGED && !vie_last_error()[0])
    set_error("not converged: a problem stopped above the tolerance (see its info)");
  return worst;
}

}  // namespace vie

using namespace vie;

namespace vie {

// Device copies of b and x for a solve on host buffers: 2 x 3N complex128,
// allocated on the plan's first such solve and kept.
static vie_status host_stage(vie_plan* p, double2** b, double2** x, int comps) {
  const size_t n3 = (size_t)comps * p->n[0] * p->n[1] * p->n[2];
  if (p->host_stage_bytes < 2 * n3 * sizeof(double2)) {
    cudaFree(p->host_stage);
    p->host_stage_bytes = 0;
    cudaError_t e = cudaMalloc(&p->host_stage, 2 * n3 * sizeof(double2));
    if (e != cudaSuccess) {
      p->host_stage = nullptr;
      set_error("staging buffers for host vectors: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA;
    }
    p->host_stage_bytes = 2 * n3 * sizeof(double2);
  }
  *b = (double2*)p->host_stage;
  *x = *b + n3;
  return VIE_OK;
}

// Solve on host buffers: copy b (and x when it is an initial guess) to the
// plans' staging buffers, solve there, copy every x back (also when the solve
// reports an error status: x then holds the last or best iterate).
static vie_status solve_host(vie_plan* const* plans, int count, const void* const* b_host, void* const* x_host,
                             double tol, const vie_solve_opts* o, vie_solve_info* infos, vie_precond_fn fn,
                             void* const* ctx, cudaStream_t s, int jm = 0) {
  const int comps = jm ? 6 : 3;
  std::vector<const double2*> bd(count);
  std::vector<double2*> xd(count);
  for (int i = 0; i < count; ++i) {
    double2* b = nullptr;
    double2* x = nullptr;
    vie_status st = host_stage(plans[i], &b, &x, comps);
    if (st != VIE_OK) return st;
    const size_t bytes = (size_t)comps * plans[i]->n[0] * plans[i]->n[1] * plans[i]->n[2] * sizeof(double2);
    VIE_CUDA_TRY(cudaMemcpyAsync(b, b_host[i], bytes, cudaMemcpyHostToDevice, s));
    if (o->x0_given) VIE_CUDA_TRY(cudaMemcpyAsync(x, x_host[i], bytes, cudaMemcpyHostToDevice, s));
    bd[i] = b;
    xd[i] = x;
  }
  vie_status st = solve_batch_impl(plans, count, bd.data(), xd.data(), tol, o, infos, fn, ctx, s, jm);
  if (st == VIE_ERR_INVALID || st == VIE_ERR_OOM || st == VIE_ERR_CUDA) return st;
  for (int i = 0; i < count; ++i) {
    const size_t bytes = (size_t)comps * plans[i]->n[0] * plans[i]->n[1] * plans[i]->n[2] * sizeof(double2);
    VIE_CUDA_TRY(cudaMemcpyAsync(x_host[i], xd[i], bytes, cudaMemcpyDeviceToHost, s));
  }
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  return st;
}

}  // namespace vie

extern "C" vie_status vie_solve(vie_plan* p, const void* b_dev, void* x_dev, double tol, const vie_solve_opts* opts,
                                vie_solve_info* info, void* stream) {
  clear_error();
  if (!p || !b_dev || !x_dev || !opts || !info) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (!(tol > 0.0 && tol < 1.0)) { set_error("tol must be in (0, 1)"); return VIE_ERR_INVALID; }
  if (opts->mode != VIE_SOLVE_FP64 && opts->mode != VIE_SOLVE_MIXED) { set_error("unknown mode"); return VIE_ERR_INVALID; }
  if (b_dev == x_dev) { set_error("b and x must differ"); return VIE_ERR_INVALID; }
  vie_precond_fn fn = nullptr;
  void* ctx = nullptr;
  if (opts->use_preconditioner) {
    vie_status st = precond_get(p, &fn, &ctx);
    if (st != VIE_OK) return st;
  }
  if (opts->host_buffers)
    return solve_host(&p, 1, &b_dev, &x_dev, tol, opts, info, fn, &ctx, (cudaStream_t)stream);
  const double2* b = (const double2*)b_dev;
  double2* x = (double2*)x_dev;
  return solve_batch_impl(&p, 1, &b, &x, tol, opts, info, fn, &ctx, (cudaStream_t)stream);
}

extern "C" vie_status vie_solve_batch(vie_plan* const* plans, int count, const void* const* b_dev,
                                      void* const* x_dev, double tol, const vie_solve_opts* opts,
                                      vie_solve_info* infos, void* stream) {
  clear_error();
  if (!plans || !b_dev || !x_dev || !opts || !infos || count < 1) {
    set_error("null argument or count < 1");
    return VIE_ERR_INVALID;
  }
  if (!(tol > 0.0 && tol < 1.0)) { set_error("tol must be in (0, 1)"); return VIE_ERR_INVALID; }
  if (opts->mode != VIE_SOLVE_FP64 && opts->mode != VIE_SOLVE_MIXED) { set_error("unknown mode"); return VIE_ERR_INVALID; }
  std::vector<void*> ctx(count, nullptr);
  vie_precond_fn fn = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || !b_dev[i] || !x_dev[i] || b_dev[i] == x_dev[i]) {
      set_error("problem %d: null plan or vector, or b == x", i);
      return VIE_ERR_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) { set_error("plan %d appears twice", i); return VIE_ERR_INVALID; }
    if (opts->use_preconditioner) {
      vie_precond_fn f = nullptr;
      vie_status st = precond_get(plans[i], &f, &ctx[i]);
      if (st != VIE_OK) return st;
      fn = f;
    }
  }
  if (opts->host_buffers)
    return solve_host(plans, count, b_dev, x_dev, tol, opts, infos, fn, ctx.data(), (cudaStream_t)stream);
  return solve_batch_impl(plans, count, (const double2* const*)b_dev, (double2* const*)x_dev, tol, opts, infos, fn,
                          ctx.data(), (cudaStream_t)stream);
}

extern "C" vie_status vie_jm_solve(vie_plan* p, const void* b, void* x, double tol, const vie_solve_opts* opts,
                                   vie_solve_info* info, void* stream) {
  clear_error();
  if (!p || !b || !x || !opts || !info) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (!(tol > 0.0 && tol < 1.0)) { set_error("tol must be in (0, 1)"); return VIE_ERR_INVALID; }
  if (opts->mode != VIE_SOLVE_FP64 && opts->mode != VIE_SOLVE_MIXED) { set_error("unknown mode"); return VIE_ERR_INVALID; }
  if (opts->use_preconditioner) { set_error("the JM-VIE solve takes no preconditioner"); return VIE_ERR_INVALID; }
  if (b == x) { set_error("b and x must differ"); return VIE_ERR_INVALID; }
  if (!p->curl) { set_error("call vie_set_permeability before a JM-VIE solve"); return VIE_ERR_INVALID; }
  if (p->jm_gen != p->contrast_gen) {
    set_error("the permittivity changed after vie_set_permeability: call it again");
    return VIE_ERR_INVALID;
  }
  void* ctx = nullptr;
  if (opts->host_buffers)
    return solve_host(&p, 1, &b, &x, tol, opts, info, nullptr, &ctx, (cudaStream_t)stream, 1);
  const double2* bd = (const double2*)b;
  double2* xd = (double2*)x;
  return solve_batch_impl(&p, 1, &bd, &xd, tol, opts, info, nullptr, &ctx, (cudaStream_t)stream, 1);
}

namespace vie {
// One grid barrier of the cooperative step in which block `absent` does not
// take part (it returns first): the other blocks' waits run out after
// `limit` clocks and set the abort word.
__global__ void barrier_probe_kernel(unsigned* bar, int absent, long long limit) {
  if ((int)blockIdx.x == absent) return;
  grid_barrier(bar, gridDim.x, limit);
}
}  // namespace vie

extern "C" vie_status vie_probe_grid_barrier(int absent_block, double wait_ms, int* aborted) {
  using namespace vie;
  clear_error();
  if (!aborted || wait_ms <= 0.0 || wait_ms > 2000.0) {
    set_error("aborted must be non-null and wait_ms in (0, 2000]");
    return VIE_ERR_INVALID;
  }
  int dev = 0, sms = 0, clk_khz = 0, coop = 0;
  VIE_CUDA_TRY(cudaGetDevice(&dev));
  VIE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VIE_CUDA_TRY(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
  VIE_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) {
    set_error("cooperative launch is not available on this device");
    return VIE_ERR_INVALID;
  }
  if (absent_block >= sms) {
    set_error("absent_block must be below the number of SMs (%d)", sms);
    return VIE_ERR_INVALID;
  }
  unsigned* bar = nullptr;
  VIE_CUDA_TRY(cudaMalloc((void**)&bar, 4 * sizeof(unsigned)));
  cudaMemset(bar, 0, 4 * sizeof(unsigned));
  const long long limit = (long long)(wait_ms * (double)clk_khz);   // clk_khz clocks per ms
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)sms);
  cfg.blockDim = dim3(32);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, barrier_probe_kernel, bar, absent_block, limit);
  unsigned h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaFree(bar);
  if (e != cudaSuccess) {
    set_error("barrier probe: %s", cudaGetErrorString(e));
    return VIE_ERR_CUDA;
  }
  *aborted = h ? 1 : 0;
  return VIE_OK;
}
