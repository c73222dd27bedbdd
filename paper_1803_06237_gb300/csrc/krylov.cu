// Krylov solvers for the discrete J-VIE (I - M_eps N) w = b (Sec. 6 of
// arXiv:1803.06237; the paper solves it with GMRES at tolerance 1e-8, Sec. 5).
//
// * Arnoldi with classical Gram-Schmidt applied twice (CGS2); dot products and
//   norms accumulate in FP64 whatever the vector type; the Hessenberg matrix,
//   Givens rotations and the small least-squares problem are FP64 and stay on
//   the device.  The host only reads a small status record every few
//   iterations.
// * Right-preconditioned flexible GMRES keeps z_j = P(v_j) (a nonlinear P is
//   allowed); with no preconditioner z_j = v_j and Z aliases V.
// * Mixed precision: iterative refinement whose residual r = b - A x uses the
//   complex128 operator and whose correction solves A d = r with the
//   complex64 operator to a loose tolerance; x accumulates in complex128.
//   Plain mode runs GMRES on the complex128 operator.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

constexpr int kDotBlocks = 456;     // 3 x 152 SMs
constexpr int kThreads = 256;

struct SolveStatus {
  int active;        // 1 while the cycle should continue
  int j;             // Arnoldi steps completed in this cycle
  int converged;     // residual estimate reached the target
  int breakdown;     // h_{j+1,j} == 0 (exact solution in the subspace) or non-finite
  double beta;       // ||r0|| of the cycle
  double target;     // absolute residual target of the cycle
  double resid;      // |g_{j+1}| (current residual estimate)
  double inv_h;      // 1 / h_{j+1,j}
};

template <typename V> __device__ __forceinline__ double2 to_d2(V v) { return make_double2((double)v.x, (double)v.y); }
template <typename V> __device__ __forceinline__ V from_d2(double2 v);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partial[i * nblk + b] = sum over block b's chunk of conj(V_i[k]) w[k], i < nv.
template <typename V>
__global__ void __launch_bounds__(kThreads) dots_kernel(const V* __restrict__ Vb, size_t ld, int nv,
                                                        const V* __restrict__ w, size_t n,
                                                        double2* __restrict__ partial,
                                                        const SolveStatus* __restrict__ st) {
  if (st && !st->active) return;
  const int nblk = gridDim.x;
  const size_t chunk = (n + nblk - 1) / nblk;
  const size_t k0 = (size_t)blockIdx.x * chunk;
  const size_t k1 = min(n, k0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < nv; i += nw) {
    const V* vi = Vb + (size_t)i * ld;
    double re = 0.0, im = 0.0;
    for (size_t k = k0 + lane; k < k1; k += 32) {
      const double2 a = to_d2(vi[k]);
      const double2 b = to_d2(w[k]);
      re += a.x * b.x + a.y * b.y;
      im += a.x * b.y - a.y * b.x;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) partial[(size_t)i * nblk + blockIdx.x] = make_double2(re, im);
  }
}

// out[i] = sum_b partial[i * nblk + b] in a fixed order (deterministic); if
// acc is given, acc[i] += out[i] as well.
__global__ void reduce_partials_kernel(const double2* __restrict__ partial, int nblk, double2* __restrict__ out,
                                       double2* __restrict__ acc, const SolveStatus* __restrict__ st) {
  if (st && !st->active) return;
  const int i = blockIdx.x;
  __shared__ double sre[kThreads], sim[kThreads];
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    re += partial[(size_t)i * nblk + b].x;
    im += partial[(size_t)i * nblk + b].y;
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
    out[i] = make_double2(sre[0], sim[0]);
    if (acc) {
      acc[i].x += sre[0];
      acc[i].y += sim[0];
    }
  }
}

// w[k] -= sum_{i<nv} V_i[k] h[i]   (FP64 accumulation)
template <typename V>
__global__ void __launch_bounds__(kThreads) update_kernel(const V* __restrict__ Vb, size_t ld, int nv,
                                                          const double2* __restrict__ h, V* __restrict__ w,
                                                          size_t n, const SolveStatus* __restrict__ st) {
  if (st && !st->active) return;
  extern __shared__ double2 hs[];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double2 acc = to_d2(w[k]);
    for (int i = 0; i < nv; ++i) {
      const double2 v = to_d2(Vb[(size_t)i * ld + k]);
      acc.x -= v.x * hs[i].x - v.y * hs[i].y;
      acc.y -= v.x * hs[i].y + v.y * hs[i].x;
    }
    w[k] = from_d2<V>(acc);
  }
}

// partial[b] = sum over chunk |w[k]|^2  (stored in .x)
template <typename V>
__global__ void __launch_bounds__(kThreads) norm2_kernel(const V* __restrict__ w, size_t n,
                                                         double2* __restrict__ partial,
                                                         const SolveStatus* __restrict__ st) {
  if (st && !st->active) return;
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const double2 a = to_d2(w[k]);
    s += a.x * a.x + a.y * a.y;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partial[blockIdx.x] = make_double2(t, 0.0);
  }
}

// dst = src * s   (types may differ; s real)
template <typename VD, typename VS>
__global__ void scale_copy_kernel(VD* __restrict__ dst, const VS* __restrict__ src, size_t n,
                                  const double* __restrict__ s_dev, double s_host,
                                  const SolveStatus* __restrict__ st, int use_inv_h) {
  if (st && !st->active) return;
  const double s = use_inv_h ? st->inv_h : (s_dev ? *s_dev : s_host);
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double2 a = to_d2(src[k]);
    a.x *= s;
    a.y *= s;
    dst[k] = from_d2<VD>(a);
  }
}

// One thread: finish Arnoldi column j (h = h1 + h2 already summed into hcol),
// apply the previous rotations, form the new one, update g and the status.
__global__ void arnoldi_step_kernel(double2* __restrict__ H, int ldh, double2* __restrict__ hcol,
                                    const double2* __restrict__ norm_partial, int nblk, double* __restrict__ cs,
                                    double2* __restrict__ sn, double2* __restrict__ g, int j,
                                    SolveStatus* __restrict__ st) {
  if (!st->active) return;
  double nrm2 = 0.0;
  for (int b = 0; b < nblk; ++b) nrm2 += norm_partial[b].x;
  const double hn = sqrt(nrm2);
  double2* col = H + (size_t)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = hcol[i];
  col[j + 1] = make_double2(hn, 0.0);
  // previous rotations
  for (int i = 0; i < j; ++i) {
    const double c = cs[i];
    const double2 s = sn[i];
    const double2 a = col[i], b = col[i + 1];
    // t = c a + s b ; b' = -conj(s) a + c b
    const double2 t = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
    const double2 bb = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    col[i] = t;
    col[i + 1] = bb;
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
    // s = (a/|a|) conj(b) / den
    const double2 ua = make_double2(a.x / aa, a.y / aa);
    s = make_double2((ua.x * b.x + ua.y * b.y) / den, (ua.y * b.x - ua.x * b.y) / den);
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
  col[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = g[j];
  g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
  g[j] = make_double2(c * gj.x, c * gj.y);
  const double res = hypot(g[j + 1].x, g[j + 1].y);
  st->j = j + 1;
  st->resid = res;
  const bool finite = isfinite(hn) && isfinite(res);
  if (!finite) {
    st->breakdown = 1;
    st->active = 0;
    st->j = j;          // drop the non-finite column
    return;
  }
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

// Back substitution R y = g (R upper triangular in H, m columns), one block.
__global__ void backsolve_kernel(const double2* __restrict__ H, int ldh, const double2* __restrict__ g,
                                 double2* __restrict__ y, const SolveStatus* __restrict__ st) {
  const int m = st->j;
  __shared__ double2 ys[1024];
  for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = g[i];
  __syncthreads();
  for (int i = m - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      const double2 r = H[(size_t)i * ldh + i];
      const double2 v = ys[i];
      const double d = r.x * r.x + r.y * r.y;
      ys[i] = make_double2((v.x * r.x + v.y * r.y) / d, (v.y * r.x - v.x * r.y) / d);
    }
    __syncthreads();
    const double2 yi = ys[i];
    for (int k = threadIdx.x; k < i; k += blockDim.x) {
      const double2 r = H[(size_t)i * ldh + k];
      ys[k].x -= r.x * yi.x - r.y * yi.y;
      ys[k].y -= r.x * yi.y + r.y * yi.x;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = ys[i];
}

// x[k] += scale * sum_{i<m} Z_i[k] y_i  (x complex128, FP64 accumulation)
template <typename V>
__global__ void __launch_bounds__(kThreads) update_x_kernel(double2* __restrict__ x, const V* __restrict__ Zb,
                                                            size_t ld, const double2* __restrict__ y,
                                                            const SolveStatus* __restrict__ st, size_t n,
                                                            double scale_) {
  extern __shared__ double2 ys[];
  const int m = st->j;
  for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < m; ++i) {
      const double2 z = to_d2(Zb[(size_t)i * ld + k]);
      acc.x += z.x * ys[i].x - z.y * ys[i].y;
      acc.y += z.x * ys[i].y + z.y * ys[i].x;
    }
    x[k].x += scale_ * acc.x;
    x[k].y += scale_ * acc.y;
  }
}

// r = b - y (complex128) with norm partials of r
__global__ void __launch_bounds__(kThreads) residual_kernel(const double2* __restrict__ b,
                                                            const double2* __restrict__ y,
                                                            double2* __restrict__ r, size_t n,
                                                            double2* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const double2 v = make_double2(b[k].x - y[k].x, b[k].y - y[k].y);
    r[k] = v;
    s += v.x * v.x + v.y * v.y;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partial[blockIdx.x] = make_double2(t, 0.0);
  }
}

__global__ void init_cycle_kernel(SolveStatus* st, double2* g, int m, double beta, double target) {
  st->active = 1;
  st->j = 0;
  st->converged = 0;
  st->breakdown = 0;
  st->beta = beta;
  st->target = target;
  st->resid = beta;
  st->inv_h = 0.0;
  for (int i = 0; i <= m; ++i) g[i] = make_double2(0.0, 0.0);
  g[0] = make_double2(beta, 0.0);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct KrylovWork {
  int m = 0;
  int dtype = 0;
  bool flexible = false;
  size_t n = 0;
  void* V = nullptr;          // (m + 1) vectors
  void* Z = nullptr;          // m vectors (flexible only)
  void* w = nullptr;          // 1 vector (same type)
  double2* x64 = nullptr;     // solution accumulator / r / y (complex128)
  double2* r64 = nullptr;
  double2* y64 = nullptr;
  double2* H = nullptr;       // (m + 1) x m, column-major, ld = m + 1
  double2* hcol = nullptr;
  double2* h2 = nullptr;
  double2* g = nullptr;
  double2* ysol = nullptr;
  double* cs = nullptr;
  double2* sn = nullptr;
  double2* partial = nullptr; // (m + 1) * kDotBlocks
  SolveStatus* st = nullptr;
  SolveStatus* st_host = nullptr;   // pinned
};

static void free_work(KrylovWork* k) {
  cudaFree(k->V); cudaFree(k->Z); cudaFree(k->w); cudaFree(k->x64); cudaFree(k->r64); cudaFree(k->y64);
  cudaFree(k->H); cudaFree(k->hcol); cudaFree(k->h2); cudaFree(k->g); cudaFree(k->ysol); cudaFree(k->cs); cudaFree(k->sn);
  cudaFree(k->partial); cudaFree(k->st); cudaFreeHost(k->st_host);
  *k = KrylovWork();
}

static vie_status alloc_work(KrylovWork* k, size_t n, int m, int dtype, bool flexible) {
  const size_t es = dtype == VIE_C64 ? sizeof(float2) : sizeof(double2);
  k->m = m; k->dtype = dtype; k->flexible = flexible; k->n = n;
  struct { void** p; size_t sz; } a[] = {
      {&k->V, (size_t)(m + 1) * n * es}, {&k->w, n * es}, {(void**)&k->x64, n * sizeof(double2)},
      {(void**)&k->r64, n * sizeof(double2)}, {(void**)&k->y64, n * sizeof(double2)},
      {(void**)&k->H, (size_t)(m + 1) * m * sizeof(double2)}, {(void**)&k->hcol, (m + 1) * sizeof(double2)}, {(void**)&k->h2, (m + 1) * sizeof(double2)},
      {(void**)&k->g, (m + 1) * sizeof(double2)}, {(void**)&k->ysol, (m + 1) * sizeof(double2)},
      {(void**)&k->cs, (m + 1) * sizeof(double)}, {(void**)&k->sn, (m + 1) * sizeof(double2)},
      {(void**)&k->partial, (size_t)(m + 2) * kDotBlocks * sizeof(double2)},
      {(void**)&k->st, sizeof(SolveStatus)}};
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
  if (cudaMallocHost((void**)&k->st_host, sizeof(SolveStatus)) != cudaSuccess) {
    set_error("cudaMallocHost failed");
    free_work(k);
    return VIE_ERR_OOM;
  }
  return VIE_OK;
}

static unsigned grid_for(size_t n) {
  const size_t b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < (size_t)152 * 8 ? b : (size_t)152 * 8);
}

static vie_status norm_host(const double2* partial_dev, int nblk, double* out, cudaStream_t s) {
  std::vector<double2> h(nblk);
  VIE_CUDA_TRY(cudaMemcpyAsync(h.data(), partial_dev, nblk * sizeof(double2), cudaMemcpyDeviceToHost, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  double t = 0.0;
  for (int i = 0; i < nblk; ++i) t += h[i].x;
  *out = sqrt(t);
  return VIE_OK;
}

// One GMRES cycle of at most m steps on the operator of type V, started from
// r (complex128, norm beta): V_0 = r / beta; stops at |g| <= target.  Adds
// beta_scale * Z y to x (complex128).  Returns the steps taken.
template <typename V>
static vie_status gmres_cycle(vie_plan* p, KrylovWork& k, int dtype, double beta, double target, int max_steps,
                              int check_every, const vie_precond_fn precond, void* precond_ctx, int* steps,
                              int* matvecs, SolveStatus* out_status, cudaStream_t s) {
  const size_t n = k.n;
  const int m = k.m;
  V* Vb = (V*)k.V;
  V* w = (V*)k.w;
  V* Zb = k.flexible ? (V*)k.Z : Vb;
  init_cycle_kernel<<<1, 1, 0, s>>>(k.st, k.g, m, beta, target);
  scale_copy_kernel<V, double2><<<grid_for(n), kThreads, 0, s>>>(Vb, k.r64, n, nullptr, 1.0 / beta, nullptr, 0);
  VIE_LAUNCH_CHECK();
  int j = 0;
  *matvecs = 0;
  const int jmax = max_steps < m ? max_steps : m;
  for (; j < jmax; ++j) {
    V* vj = Vb + (size_t)j * n;
    V* zj = Zb + (size_t)j * n;
    if (k.flexible) {
      vie_status ps = precond(precond_ctx, dtype, vj, zj, s);
      if (ps != VIE_OK) return ps;
    }
    vie_status ms = matvec_impl(p, zj, w, dtype, MODE_OPERATOR, p->work, s);
    if (ms != VIE_OK) return ms;
    ++*matvecs;
    const int nv = j + 1;
    // CGS2: h1 = V^H w, w -= V h1; h2 = V^H w, w -= V h2; column = h1 + h2
    dots_kernel<V><<<kDotBlocks, kThreads, 0, s>>>(Vb, n, nv, w, n, k.partial, k.st);
    reduce_partials_kernel<<<nv, kThreads, 0, s>>>(k.partial, kDotBlocks, k.hcol, nullptr, k.st);
    update_kernel<V><<<grid_for(n), kThreads, nv * sizeof(double2), s>>>(Vb, n, nv, k.hcol, w, n, k.st);
    dots_kernel<V><<<kDotBlocks, kThreads, 0, s>>>(Vb, n, nv, w, n, k.partial, k.st);
    reduce_partials_kernel<<<nv, kThreads, 0, s>>>(k.partial, kDotBlocks, k.h2, k.hcol, k.st);
    update_kernel<V><<<grid_for(n), kThreads, nv * sizeof(double2), s>>>(Vb, n, nv, k.h2, w, n, k.st);
    VIE_LAUNCH_CHECK();
    norm2_kernel<V><<<kDotBlocks, kThreads, 0, s>>>(w, n, k.partial, k.st);
    arnoldi_step_kernel<<<1, 1, 0, s>>>(k.H, m + 1, k.hcol, k.partial, kDotBlocks, k.cs, k.sn, k.g, j, k.st);
    scale_copy_kernel<V, V><<<grid_for(n), kThreads, 0, s>>>(Vb + (size_t)(j + 1) * n, w, n, nullptr, 0.0, k.st, 1);
    VIE_LAUNCH_CHECK();
    if ((j + 1) % check_every == 0 || j + 1 == jmax) {
      VIE_CUDA_TRY(cudaMemcpyAsync(k.st_host, k.st, sizeof(SolveStatus), cudaMemcpyDeviceToHost, s));
      VIE_CUDA_TRY(cudaStreamSynchronize(s));
      if (!k.st_host->active) break;
    }
  }
  VIE_CUDA_TRY(cudaMemcpyAsync(k.st_host, k.st, sizeof(SolveStatus), cudaMemcpyDeviceToHost, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  *steps = k.st_host->j;
  *out_status = *k.st_host;
  if (*steps > 0) {
    backsolve_kernel<<<1, 256, 0, s>>>(k.H, m + 1, k.g, k.ysol, k.st);
    update_x_kernel<V><<<grid_for(n), kThreads, (size_t)m * sizeof(double2), s>>>(k.x64, Zb, n, k.ysol, k.st, n, 1.0);
    VIE_LAUNCH_CHECK();
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

static vie_status ensure_work(vie_plan* p, int m, int dtype, bool flexible, KrylovWork** out) {
  const size_t n = (size_t)3 * p->n[0] * p->n[1] * p->n[2];
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

// true residual r = b - A64 x into k.r64; returns ||r||
static vie_status true_residual(vie_plan* p, KrylovWork& k, const double2* b, double* rnorm, cudaStream_t s) {
  vie_status st = matvec_impl(p, k.x64, k.y64, VIE_C128, MODE_OPERATOR, p->work, s);
  if (st != VIE_OK) return st;
  residual_kernel<<<kDotBlocks, kThreads, 0, s>>>(b, k.y64, k.r64, k.n, k.partial);
  VIE_LAUNCH_CHECK();
  return norm_host(k.partial, kDotBlocks, rnorm, s);
}

vie_status solve_impl(vie_plan* p, const double2* b, double2* x, double tol, const vie_solve_opts* o,
                      vie_solve_info* info, vie_precond_fn precond, void* precond_ctx, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const int mode = o->mode;
  const int m = o->restart > 0 ? o->restart : 100;
  if (m > 1000) { set_error("restart must be <= 1000"); return VIE_ERR_INVALID; }
  const int max_iters = o->max_iters > 0 ? o->max_iters : 5000;
  const int max_outer = o->max_outer > 0 ? o->max_outer : 200;
  const double inner_tol = o->inner_tol > 0 ? o->inner_tol : 1e-4;
  const int check_every = o->check_every > 0 ? o->check_every : 4;
  const double timeout = o->timeout_s > 0 ? o->timeout_s : 600.0;
  const int dtype = (mode == VIE_SOLVE_MIXED) ? VIE_C64 : VIE_C128;
  const bool flexible = precond != nullptr;
  KrylovWork* kp = nullptr;
  vie_status st = ensure_work(p, m, dtype, flexible, &kp);
  if (st != VIE_OK) return st;
  KrylovWork& k = *kp;
  const size_t n = k.n;
  memset(info, 0, sizeof(*info));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  // ||b||
  norm2_kernel<double2><<<kDotBlocks, kThreads, 0, s>>>(b, n, k.partial, nullptr);
  VIE_LAUNCH_CHECK();
  double bnorm = 0.0;
  st = norm_host(k.partial, kDotBlocks, &bnorm, s);
  if (st != VIE_OK) return st;
  if (!isfinite(bnorm)) { set_error("right-hand side is not finite"); return VIE_ERR_NONFINITE; }
  if (o->x0_given) {
    VIE_CUDA_TRY(cudaMemcpyAsync(k.x64, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  } else {
    VIE_CUDA_TRY(cudaMemsetAsync(k.x64, 0, n * sizeof(double2), s));
  }
  if (bnorm == 0.0) {
    VIE_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
    info->converged = 1;
    VIE_CUDA_TRY(cudaStreamSynchronize(s));
    return VIE_OK;
  }
  int iters = 0, outer = 0;
  double rnorm = 0.0;
  bool converged = false;
  st = VIE_OK;
  while (true) {
    st = true_residual(p, k, b, &rnorm, s);
    if (st != VIE_OK) break;
    info->matvecs64++;
    if (outer < (int)(sizeof(info->history) / sizeof(info->history[0]))) info->history[outer] = rnorm / bnorm;
    info->history_len = outer + 1;
    if (!isfinite(rnorm)) { set_error("residual became non-finite"); st = VIE_ERR_NONFINITE; break; }
    if (rnorm <= tol * bnorm) { converged = true; break; }
    if (iters >= max_iters || outer >= max_outer) break;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (secs > timeout) { set_error("solve exceeded %.1f s", timeout); st = VIE_ERR_TIMEOUT; break; }
    // inner target: plain mode goes straight for tol (absolute tol * ||b||);
    // mixed mode asks the complex64 cycle for a relative reduction inner_tol,
    // never below what the outer target needs.
    double target = tol * bnorm;
    if (mode == VIE_SOLVE_MIXED) target = fmax(inner_tol * rnorm, 0.5 * tol * bnorm);
    int steps = 0, mv = 0;
    SolveStatus cs;
    if (dtype == VIE_C64)
      st = gmres_cycle<float2>(p, k, dtype, rnorm, target, max_iters - iters, check_every, precond, precond_ctx,
                               &steps, &mv, &cs, s);
    else
      st = gmres_cycle<double2>(p, k, dtype, rnorm, target, max_iters - iters, check_every, precond, precond_ctx,
                                &steps, &mv, &cs, s);
    if (st != VIE_OK) break;
    iters += steps;
    outer++;
    if (dtype == VIE_C64) info->matvecs32 += mv; else info->matvecs64 += mv;
    if (steps == 0) { set_error("Krylov cycle made no progress (breakdown at the first step)"); break; }
  }
  cudaEventRecord(e1, s);
  if (st == VIE_OK || st == VIE_ERR_TIMEOUT) {
    cudaError_t e = cudaMemcpyAsync(x, k.x64, n * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == VIE_OK) { set_error("copy-out failed: %s", cudaGetErrorString(e)); st = VIE_ERR_CUDA; }
  }
  float ms = 0.f;
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  info->iterations = iters;
  info->outer = outer;
  info->residual = rnorm / bnorm;
  info->converged = converged ? 1 : 0;
  info->time_ms = ms;
  if (st == VIE_OK && !converged) {
    if (!vie_last_error()[0]) set_error("not converged: relative residual %.3e after %d iterations", rnorm / bnorm, iters);
    return VIE_ERR_NOT_CONVERGED;
  }
  return st;
}

}  // namespace vie

extern "C" vie_status vie_solve(vie_plan* p, const void* b_dev, void* x_dev, double tol, const vie_solve_opts* opts,
                                vie_solve_info* info, void* stream) {
  vie::clear_error();
  if (!p || !b_dev || !x_dev || !opts || !info) { vie::set_error("null argument"); return VIE_ERR_INVALID; }
  if (!(tol > 0.0 && tol < 1.0)) { vie::set_error("tol must be in (0, 1)"); return VIE_ERR_INVALID; }
  if (opts->mode != VIE_SOLVE_FP64 && opts->mode != VIE_SOLVE_MIXED) { vie::set_error("unknown mode"); return VIE_ERR_INVALID; }
  if (b_dev == x_dev) { vie::set_error("b and x must differ"); return VIE_ERR_INVALID; }
  vie::vie_precond_fn fn = nullptr;
  void* ctx = nullptr;
  if (opts->use_preconditioner) {
    vie_status st = vie::precond_get(p, &fn, &ctx);
    if (st != VIE_OK) return st;
  }
  return vie::solve_impl(p, (const double2*)b_dev, (double2*)x_dev, tol, opts, info, fn, ctx, (cudaStream_t)stream);
}
