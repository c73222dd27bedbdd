// Setup on the device, in FP64: Galerkin Toeplitz entries of N and the
// spectra of their circulant embedding.
//
// Paper (arXiv:1803.06237): N f = curl curl S f with G = exp(-j k r)/(4 pi r)
// (Sec. 3); N_ij = <N P_j, P_i> with P_i = h^(-3/2) on voxel i (Sec. 3.1);
// N is block-Toeplitz with six unique tensor components and its product is
// computed with FFTs (Sec. 5.4).
//
// With h as the unit of length and kappa = k h, (lap + k^2) G = -delta gives
// N = k^2 S + grad div S + I, and the entry for offset D and components p, q is
//   T_pq(D) = delta_pq delta_D0 + int L_D(v) (kappa^2 delta_pq + d_p d_q) g(v) dv,
// L_D(v) = prod_a max(0, 1 - |v_a - D_a|) (the overlap of two unit voxels),
// g(v) = exp(-j kappa |v|)/(4 pi |v|), the derivatives taken in the sense of
// distributions.  Two routes are used:
//   * |D|_inf >= 2: the support of L_D misses v = 0, so the derivatives act on g
//     (closed-form dyadic kernel) and the tent-weighted integral is done with
//     tensor Gauss-Legendre over the 8 unit cells of the support.
//   * |D|_inf <= 1: the derivatives act on L_D.  The off-diagonal part becomes
//     int g sign(v_p - D_p) sign(v_q - D_q) L(v_r - D_r) dv, the diagonal part a
//     second difference of plane integrals F_p(t) = int int g L L over the
//     planes v_p = D_p - 1, D_p, D_p + 1.  Unit cells that have the origin as
//     a corner use the Duffy map (pyramids / triangles, Jacobian t^2 / t).
#include <math.h>
#include <stdio.h>
#include <vector>

#include "fft.cuh"
#include "vie_internal.cuh"

namespace vie {

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes on [0, 1] for orders 1..kMaxGL (host Newton iteration
// on the three-term Legendre recurrence), stored at offset q (q - 1) / 2.
// ---------------------------------------------------------------------------
constexpr int kMaxGL = 24;
__constant__ double c_gl_x[kMaxGL * (kMaxGL + 1) / 2];
__constant__ double c_gl_w[kMaxGL * (kMaxGL + 1) / 2];

static void legendre_nodes(int q, double* x01, double* w01) {
  for (int i = 0; i < q; ++i) {
    double x = cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= q; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = x; p0 = 1.0; }
      dp = q * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    // recompute the derivative at the converged node
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= q; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (q == 1) { p1 = x; p0 = 1.0; }
    dp = q * (x * p1 - p0) / (x * x - 1.0);
    x01[i] = 0.5 * (1.0 - x);
    w01[i] = 1.0 / ((1.0 - x * x) * dp * dp);   // (2/((1-x^2) P'^2)) / 2
  }
}

static vie_status upload_gl_tables() {
  static bool done[64] = {false};
  int dev = 0;
  VIE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 64 && done[dev]) return VIE_OK;
  std::vector<double> xs(kMaxGL * (kMaxGL + 1) / 2), ws(xs.size());
  for (int q = 1; q <= kMaxGL; ++q) legendre_nodes(q, &xs[q * (q - 1) / 2], &ws[q * (q - 1) / 2]);
  VIE_CUDA_TRY(cudaMemcpyToSymbol(c_gl_x, xs.data(), xs.size() * sizeof(double)));
  VIE_CUDA_TRY(cudaMemcpyToSymbol(c_gl_w, ws.data(), ws.size() * sizeof(double)));
  VIE_CUDA_TRY(cudaDeviceSynchronize());
  if (dev < 64) done[dev] = true;
  return VIE_OK;
}

__host__ __device__ inline int gl_order_for(int cheb) {
  if (cheb <= 2) return 16;
  if (cheb == 3) return 13;
  if (cheb <= 5) return 11;
  if (cheb <= 9) return 9;
  if (cheb <= 19) return 7;
  return 6;
}

constexpr int kQNear = 16;

__device__ __forceinline__ double tent(double t) { return fmax(0.0, 1.0 - fabs(t)); }
__device__ __forceinline__ double sgn1(double t) { return fabs(t) < 1.0 ? (t > 0.0 ? 1.0 : (t < 0.0 ? -1.0 : 0.0)) : 0.0; }

// g(r) * w as (re, im)
__device__ __forceinline__ double2 green_w(double r, double kappa, double w) {
  double s, c;
  sincos(kappa * r, &s, &c);
  const double f = w / (4.0 * M_PI * r);
  return make_double2(c * f, -s * f);
}

// ---------------------------------------------------------------------------
// near offsets: one block per D in {0,1}^3
// ---------------------------------------------------------------------------
// accumulator slots: 0 V, 1 xy, 2 xz, 3 yz, 4 + 3p + (dt+1) F_p(D_p + dt)
constexpr int kNearAcc = 13;

__device__ void block_reduce_acc(double2* acc, double* red, int tid, int nth) {
  // warp reduce then shared reduce; red has (nth/32) * 2 * kNearAcc doubles
  const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  for (int k = 0; k < kNearAcc; ++k) {
    double re = acc[k].x, im = acc[k].y;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) { red[(warp * kNearAcc + k) * 2] = re; red[(warp * kNearAcc + k) * 2 + 1] = im; }
  }
  __syncthreads();
  if (tid < kNearAcc) {
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nw; ++w) { re += red[(w * kNearAcc + tid) * 2]; im += red[(w * kNearAcc + tid) * 2 + 1]; }
    red[(nw * kNearAcc + tid) * 2] = re;
    red[(nw * kNearAcc + tid) * 2 + 1] = im;
  }
  __syncthreads();
}

__global__ void near_entries_kernel(double2* __restrict__ T, int nx, int ny, int nz, double kappa) {
  const int b = blockIdx.x;                    // D = (b&1, (b>>1)&1, (b>>2)&1)
  const int D[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
  if (D[0] >= nx || D[1] >= ny || D[2] >= nz) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int q = kQNear;
  const double* X = c_gl_x + q * (q - 1) / 2;
  const double* W = c_gl_w + q * (q - 1) / 2;
  double2 acc[kNearAcc];
  for (int k = 0; k < kNearAcc; ++k) acc[k] = make_double2(0.0, 0.0);

  // ---- volume: 8 unit cells covering [D-1, D+1]^3
  for (int cell = 0; cell < 8; ++cell) {
    int c0[3] = {D[0] - 1 + (cell & 1), D[1] - 1 + ((cell >> 1) & 1), D[2] - 1 + ((cell >> 2) & 1)};
    const bool duffy = (c0[0] == 0 || c0[0] == -1) && (c0[1] == 0 || c0[1] == -1) && (c0[2] == 0 || c0[2] == -1);
    const int q3 = q * q * q;
    const int npts = duffy ? 3 * q3 : q3;
    for (int pt = tid; pt < npts; pt += nth) {
      const int a = pt / q3, rest = pt - a * q3;
      const int i = rest / (q * q), j = (rest / q) % q, k = rest % q;
      double v[3], w;
      if (duffy) {
        const double t = X[i];
        double u[3];
        u[a] = t;
        u[(a + 1) % 3] = t * X[j];
        u[(a + 2) % 3] = t * X[k];
        for (int d = 0; d < 3; ++d) v[d] = (c0[d] == -1) ? -u[d] : u[d];
        w = W[i] * W[j] * W[k] * t * t;
      } else {
        v[0] = c0[0] + X[i]; v[1] = c0[1] + X[j]; v[2] = c0[2] + X[k];
        w = W[i] * W[j] * W[k];
      }
      const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      const double2 g = green_w(r, kappa, w);
      const double rx = v[0] - D[0], ry = v[1] - D[1], rz = v[2] - D[2];
      const double Lx = tent(rx), Ly = tent(ry), Lz = tent(rz);
      const double Sx = sgn1(rx), Sy = sgn1(ry), Sz = sgn1(rz);
      const double f[4] = {Lx * Ly * Lz, Sx * Sy * Lz, Sx * Sz * Ly, Sy * Sz * Lx};
      for (int s = 0; s < 4; ++s) { acc[s].x += g.x * f[s]; acc[s].y += g.y * f[s]; }
    }
  }
  // ---- planes: F_p(D_p + dt) over 4 unit squares
  for (int p = 0; p < 3; ++p) {
    const int a = (p + 1) % 3, bb = (p + 2) % 3;
    for (int dt = -1; dt <= 1; ++dt) {
      const int tp = D[p] + dt;
      for (int sq = 0; sq < 4; ++sq) {
        const int ca = D[a] - 1 + (sq & 1), cb = D[bb] - 1 + ((sq >> 1) & 1);
        const bool duffy = (tp == 0) && (ca == 0 || ca == -1) && (cb == 0 || cb == -1);
        const int q2 = q * q;
        const int npts = duffy ? 2 * q2 : q2;
        for (int pt = tid; pt < npts; pt += nth) {
          const int tri = pt / q2, rest = pt - tri * q2;
          const int i = rest / q, j = rest % q;
          double va, vb, w;
          if (duffy) {
            const double t = X[i];
            double u0 = tri == 0 ? t : t * X[j];
            double u1 = tri == 0 ? t * X[j] : t;
            va = (ca == -1) ? -u0 : u0;
            vb = (cb == -1) ? -u1 : u1;
            w = W[i] * W[j] * t;
          } else {
            va = ca + X[i];
            vb = cb + X[j];
            w = W[i] * W[j];
          }
          const double r = sqrt((double)tp * tp + va * va + vb * vb);
          const double2 g = green_w(r, kappa, w * tent(va - D[a]) * tent(vb - D[bb]));
          const int s = 4 + 3 * p + (dt + 1);
          acc[s].x += g.x;
          acc[s].y += g.y;
        }
      }
    }
  }
  extern __shared__ double red[];
  block_reduce_acc(acc, red, tid, nth);
  if (tid == 0) {
    const double* R = red + (nth >> 5) * kNearAcc * 2;
    const double2 V = make_double2(R[0], R[1]);
    const size_t N = (size_t)nx * ny * nz;
    const size_t vox = ((size_t)D[2] * ny + D[1]) * nx + D[0];
    const bool self = (D[0] | D[1] | D[2]) == 0;
    const double k2 = kappa * kappa;
    for (int p = 0; p < 3; ++p) {
      const double* F = R + 2 * (4 + 3 * p);
      double re = (self ? 1.0 : 0.0) + k2 * V.x + F[4] - 2.0 * F[2] + F[0];
      double im = k2 * V.y + F[5] - 2.0 * F[3] + F[1];
      T[p * N + vox] = make_double2(re, im);
    }
    for (int c = 0; c < 3; ++c) T[(3 + c) * N + vox] = make_double2(R[2 * (1 + c)], R[2 * (1 + c) + 1]);
  }
}

// ---------------------------------------------------------------------------
// far offsets: one warp per D with |D|_inf >= 2 (dyadic kernel, tent weight)
// ---------------------------------------------------------------------------
__global__ void far_entries_kernel(double2* __restrict__ T, int nx, int ny, int nz, double kappa) {
  const size_t N = (size_t)nx * ny * nz;
  const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= N) return;
  const int dx = (int)(gw % nx), dy = (int)((gw / nx) % ny), dz = (int)(gw / ((size_t)nx * ny));
  const int cheb = max(dx, max(dy, dz));
  if (cheb <= 1) return;
  const int q = gl_order_for(cheb);
  const double* X = c_gl_x + q * (q - 1) / 2;
  const double* W = c_gl_w + q * (q - 1) / 2;
  const int q3 = q * q * q;
  const int npts = 8 * q3;
  double acc[12];
  for (int k = 0; k < 12; ++k) acc[k] = 0.0;
  const double k2 = kappa * kappa;
  for (int pt = lane; pt < npts; pt += 32) {
    const int cell = pt / q3, rest = pt - cell * q3;
    const int i = rest / (q * q), j = (rest / q) % q, k = rest % q;
    const double ox = (cell & 1) - 1 + X[i], oy = ((cell >> 1) & 1) - 1 + X[j], oz = ((cell >> 2) & 1) - 1 + X[k];
    const double w = W[i] * W[j] * W[k] * (1.0 - fabs(ox)) * (1.0 - fabs(oy)) * (1.0 - fabs(oz));
    const double v0 = dx + ox, v1 = dy + oy, v2 = dz + oz;
    const double r2 = v0 * v0 + v1 * v1 + v2 * v2;
    const double r = sqrt(r2);
    double s, c;
    sincos(kappa * r, &s, &c);
    // e^{-j kr} / (4 pi r^3) [ (k^2 r^2 - 1 - j kr) d_pq + (3 + 3 j kr - k^2 r^2) vp vq / r^2 ]
    const double f = w / (4.0 * M_PI * r * r2);
    const double er = c * f, ei = -s * f;
    const double kr = kappa * r;
    const double ar = k2 * r2 - 1.0, ai = -kr;
    const double br = 3.0 - k2 * r2, bi = 3.0 * kr;
    const double inv_r2 = 1.0 / r2;
    const double vv[6] = {v0 * v0 * inv_r2, v1 * v1 * inv_r2, v2 * v2 * inv_r2,
                          v0 * v1 * inv_r2, v0 * v2 * inv_r2, v1 * v2 * inv_r2};
    for (int cc = 0; cc < 6; ++cc) {
      double tr = br * vv[cc], ti = bi * vv[cc];
      if (cc < 3) { tr += ar; ti += ai; }
      acc[2 * cc] += er * tr - ei * ti;
      acc[2 * cc + 1] += er * ti + ei * tr;
    }
  }
  for (int k = 0; k < 12; ++k)
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  if (lane == 0)
    for (int cc = 0; cc < 6; ++cc) T[cc * N + gw] = make_double2(acc[2 * cc], acc[2 * cc + 1]);
}

// ---------------------------------------------------------------------------
// circulant embedding of the octant: full[c][mz][my][mx]
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fold_index(int m, int n, int M, bool* neg, bool* valid) {
  if (m < n) { *neg = false; *valid = true; return m; }
  if (m > M - n) { *neg = true; *valid = true; return M - m; }
  *neg = false; *valid = false; return 0;
}

__global__ void embed_kernel(const double2* __restrict__ T, double2* __restrict__ full,
                             int nx, int ny, int nz, int Mx, int My, int Mz) {
  const size_t total = (size_t)6 * Mx * My * Mz;
  const size_t N = (size_t)nx * ny * nz;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int mx = (int)(idx % Mx);
    const int my = (int)((idx / Mx) % My);
    const int mz = (int)((idx / ((size_t)Mx * My)) % Mz);
    const int c = (int)(idx / ((size_t)Mx * My * Mz));
    bool nx_, ny_, nz_, vx, vy, vz;
    const int dx = fold_index(mx, nx, Mx, &nx_, &vx);
    const int dy = fold_index(my, ny, My, &ny_, &vy);
    const int dz = fold_index(mz, nz, Mz, &nz_, &vz);
    double2 val = make_double2(0.0, 0.0);
    if (vx && vy && vz) {
      val = T[c * N + ((size_t)dz * ny + dy) * nx + dx];
      // odd components: xy odd in x and y, xz in x and z, yz in y and z
      bool flip = false;
      if (c == 3) flip = nx_ ^ ny_;
      if (c == 4) flip = nx_ ^ nz_;
      if (c == 5) flip = ny_ ^ nz_;
      if (flip) { val.x = -val.x; val.y = -val.y; }
    }
    full[idx] = val;
  }
}

// ---------------------------------------------------------------------------
// FP64 FFT of the embedded components along one axis (forward).  Line (o, i)
// has elements at o*outer_stride + i*inner_stride + k*axis_stride, k < len.  A
// block takes `tl` consecutive inner indices of one outer index; when the axis
// is contiguous (axis_stride == 1) elements are read along k, otherwise along
// i, so that global accesses are coalesced either way.
// ---------------------------------------------------------------------------
__global__ void fft_axis_f64_kernel(double2* __restrict__ data, Radices rd, const double2* __restrict__ twg,
                                    long long n_outer, long long outer_stride, long long n_inner,
                                    long long inner_stride, long long axis_stride, int tl) {
  extern __shared__ double2 sm64[];
  const int L = rd.len;
  const int pitch = L + 1;
  double2* tw = sm64;
  double2* A = tw + L;
  double2* B = A + (size_t)tl * pitch;
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long groups_per_outer = (n_inner + tl - 1) / tl;
  const long long g = blockIdx.x;
  const long long o = g / groups_per_outer;
  const long long i0 = (g % groups_per_outer) * tl;
  if (o >= n_outer) return;
  const int nl = (int)min((long long)tl, n_inner - i0);
  double2* base = data + o * outer_stride + i0 * inner_stride;
  const bool contig = (axis_stride == 1);
  for (int i = tid; i < L; i += nth) tw[i] = twg[i];
  for (int e = tid; e < nl * L; e += nth) {
    int k, l;
    if (contig) { l = e / L; k = e - l * L; } else { k = e / nl; l = e - k * nl; }
    A[l * pitch + k] = base[l * inner_stride + k * axis_stride];
  }
  __syncthreads();
  double2* res = fft_lines<double2, false>(A, B, rd, pitch, nl, tw, tid, nth);
  for (int e = tid; e < nl * L; e += nth) {
    int k, l;
    if (contig) { l = e / L; k = e - l * L; } else { k = e / nl; l = e - k * nl; }
    base[l * inner_stride + k * axis_stride] = res[l * pitch + k];
  }
}

// ---------------------------------------------------------------------------
// fold to the octant, scale by 1/(Mx My Mz), layout [kx'][c][kz'][ky']
// ---------------------------------------------------------------------------
__global__ void fold_spectrum_kernel(const double2* __restrict__ full, double2* __restrict__ g64,
                                     float2* __restrict__ g32, int Mx, int My, int Mz,
                                     int Kx, int Ky, int Kz, double scale_) {
  const size_t total = (size_t)Kx * 6 * Kz * Ky;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(idx % Ky);
    const int kz = (int)((idx / Ky) % Kz);
    const int c = (int)((idx / ((size_t)Ky * Kz)) % 6);
    const int kx = (int)(idx / ((size_t)Ky * Kz * 6));
    double2 v = full[(((size_t)c * Mz + kz) * My + ky) * Mx + kx];
    v.x *= scale_;
    v.y *= scale_;
    g64[idx] = v;
    g32[idx] = make_float2((float)v.x, (float)v.y);
  }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
vie_status compute_toeplitz(vie_plan* p, cudaStream_t s) {
  vie_status st = upload_gl_tables();
  if (st != VIE_OK) return st;
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const size_t N = (size_t)nx * ny * nz;
  {
    const int threads = 256;
    const size_t warps = N;
    const size_t blocks = (warps * 32 + threads - 1) / threads;
    far_entries_kernel<<<(unsigned)blocks, threads, 0, s>>>(p->toeplitz, nx, ny, nz, p->kappa);
    VIE_LAUNCH_CHECK();
  }
  {
    const int threads = 256;
    const size_t smem = (size_t)(threads / 32 + 1) * kNearAcc * 2 * sizeof(double);
    near_entries_kernel<<<8, threads, smem, s>>>(p->toeplitz, nx, ny, nz, p->kappa);
    VIE_LAUNCH_CHECK();
  }
  return VIE_OK;
}

static vie_status fft_axis_f64(double2* data, const AxisPlan& ax, long long n_outer, long long outer_stride,
                               long long n_inner, long long inner_stride, long long axis_stride,
                               cudaStream_t s) {
  const int L = ax.len;
  const size_t per_line = (size_t)2 * (L + 1) * sizeof(double2);
  const size_t tw_bytes = (size_t)L * sizeof(double2);
  const size_t budget = 200 * 1024;
  if (tw_bytes + per_line > budget) {
    set_error("FFT length %d too large for the setup transform", L);
    return VIE_ERR_INVALID;
  }
  int tl = 8;
  while (tl > 1 && tw_bytes + (size_t)tl * per_line > budget) tl >>= 1;
  const size_t smem = tw_bytes + (size_t)tl * per_line;
  VIE_CUDA_TRY(cudaFuncSetAttribute(fft_axis_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long groups = n_outer * ((n_inner + tl - 1) / tl);
  fft_axis_f64_kernel<<<(unsigned)groups, 256, smem, s>>>(data, radices_of(ax), ax.tw64, n_outer, outer_stride,
                                                          n_inner, inner_stride, axis_stride, tl);
  VIE_LAUNCH_CHECK();
  return VIE_OK;
}

vie_status compute_spectrum(vie_plan* p, cudaStream_t s) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int Mx = p->m[0], My = p->m[1], Mz = p->m[2];
  const size_t cells = (size_t)Mx * My * Mz;
  double2* full = nullptr;
  VIE_CUDA_TRY(cudaMallocAsync((void**)&full, 6 * cells * sizeof(double2), s));
  vie_status st = VIE_OK;
  {
    const size_t total = 6 * cells;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    embed_kernel<<<blocks, 256, 0, s>>>(p->toeplitz, full, nx, ny, nz, Mx, My, Mz);
    if (cudaGetLastError() != cudaSuccess) { set_error("embed_kernel launch failed"); st = VIE_ERR_CUDA; }
  }
  // x: contiguous rows (6 Mz My of them)
  if (st == VIE_OK) st = fft_axis_f64(full, p->ax[0], 1, 0, 6LL * Mz * My, Mx, 1, s);
  // y: outer (c, mz), inner mx, axis stride Mx
  if (st == VIE_OK) st = fft_axis_f64(full, p->ax[1], 6LL * Mz, (long long)My * Mx, Mx, 1, Mx, s);
  // z: outer c, inner (my, mx), axis stride My Mx
  if (st == VIE_OK) st = fft_axis_f64(full, p->ax[2], 6, (long long)Mz * My * Mx, (long long)My * Mx, 1,
                                      (long long)My * Mx, s);
  if (st == VIE_OK) {
    const size_t total = (size_t)p->kf[0] * 6 * p->kf[2] * p->kf[1];
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    fold_spectrum_kernel<<<blocks, 256, 0, s>>>(full, p->ghat64, p->ghat32, Mx, My, Mz, p->kf[0], p->kf[1],
                                                p->kf[2], 1.0 / (double)cells);
    if (cudaGetLastError() != cudaSuccess) { set_error("fold_spectrum_kernel launch failed"); st = VIE_ERR_CUDA; }
  }
  cudaError_t e = cudaFreeAsync(full, s);
  if (st == VIE_OK && e != cudaSuccess) { set_error("cudaFreeAsync: %s", cudaGetErrorString(e)); st = VIE_ERR_CUDA; }
  return st;
}

// ---------------------------------------------------------------------------
// JM-VIE (Sec. 3): Galerkin entries of the scalar derivatives of S, in units
// of h, C_a(D) = <P_i, d_a S P_j> / h = int (d_a g)(v) L_D(v) dv; the curl
// operator K = curl S has K_pq(D) = h eps_paq C_a(D).  C_a is odd in D_a and
// even in the other two offsets, C_a(0) = 0.  As for T:
//   * |D|_inf >= 2: d_a g in closed form, -g (1 + j kappa r) v_a / r^2, with
//     the tent weight, tensor Gauss-Legendre over the 8 unit cells;
//   * |D|_inf = 1: by parts on the tent, C_a = int g sign(v_a - D_a)
//     L(v_b - D_b) L(v_c - D_c) dv, Duffy cells where the origin is a corner.
// Stored like T: octant [a][z][y][x] for D in [0, n).
// ---------------------------------------------------------------------------
__global__ void near_curl_kernel(double2* __restrict__ C, int nx, int ny, int nz, double kappa) {
  const int b = blockIdx.x;                    // D = (b&1, (b>>1)&1, (b>>2)&1), D != 0
  const int D[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
  if (D[0] >= nx || D[1] >= ny || D[2] >= nz) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int q = kQNear;
  const double* X = c_gl_x + q * (q - 1) / 2;
  const double* W = c_gl_w + q * (q - 1) / 2;
  double2 acc[kNearAcc];
  for (int k = 0; k < kNearAcc; ++k) acc[k] = make_double2(0.0, 0.0);
  if (b != 0) {
    for (int cell = 0; cell < 8; ++cell) {
      int c0[3] = {D[0] - 1 + (cell & 1), D[1] - 1 + ((cell >> 1) & 1), D[2] - 1 + ((cell >> 2) & 1)};
      const bool duffy = (c0[0] == 0 || c0[0] == -1) && (c0[1] == 0 || c0[1] == -1) && (c0[2] == 0 || c0[2] == -1);
      const int q3 = q * q * q;
      const int npts = duffy ? 3 * q3 : q3;
      for (int pt = tid; pt < npts; pt += nth) {
        const int a = pt / q3, rest = pt - a * q3;
        const int i = rest / (q * q), j = (rest / q) % q, k = rest % q;
        double v[3], w;
        if (duffy) {
          const double t = X[i];
          double u[3];
          u[a] = t;
          u[(a + 1) % 3] = t * X[j];
          u[(a + 2) % 3] = t * X[k];
          for (int d = 0; d < 3; ++d) v[d] = (c0[d] == -1) ? -u[d] : u[d];
          w = W[i] * W[j] * W[k] * t * t;
        } else {
          v[0] = c0[0] + X[i]; v[1] = c0[1] + X[j]; v[2] = c0[2] + X[k];
          w = W[i] * W[j] * W[k];
        }
        const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const double2 g = green_w(r, kappa, w);
        const double rx = v[0] - D[0], ry = v[1] - D[1], rz = v[2] - D[2];
        const double Lx = tent(rx), Ly = tent(ry), Lz = tent(rz);
        const double f[3] = {sgn1(rx) * Ly * Lz, Lx * sgn1(ry) * Lz, Lx * Ly * sgn1(rz)};
        for (int s = 0; s < 3; ++s) { acc[s].x += g.x * f[s]; acc[s].y += g.y * f[s]; }
      }
    }
  }
  extern __shared__ double red[];
  block_reduce_acc(acc, red, tid, nth);
  if (tid == 0) {
    const double* R = red + (nth >> 5) * kNearAcc * 2;
    const size_t N = (size_t)nx * ny * nz;
    const size_t vox = ((size_t)D[2] * ny + D[1]) * nx + D[0];
    for (int a = 0; a < 3; ++a) C[a * N + vox] = make_double2(R[2 * a], R[2 * a + 1]);
  }
}

__global__ void far_curl_kernel(double2* __restrict__ C, int nx, int ny, int nz, double kappa) {
  const size_t N = (size_t)nx * ny * nz;
  const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= N) return;
  const int dx = (int)(gw % nx), dy = (int)((gw / nx) % ny), dz = (int)(gw / ((size_t)nx * ny));
  const int cheb = max(dx, max(dy, dz));
  if (cheb <= 1) return;
  const int q = gl_order_for(cheb);
  const double* X = c_gl_x + q * (q - 1) / 2;
  const double* W = c_gl_w + q * (q - 1) / 2;
  const int q3 = q * q * q;
  const int npts = 8 * q3;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int pt = lane; pt < npts; pt += 32) {
    const int cell = pt / q3, rest = pt - cell * q3;
    const int i = rest / (q * q), j = (rest / q) % q, k = rest % q;
    const double ox = (cell & 1) - 1 + X[i], oy = ((cell >> 1) & 1) - 1 + X[j], oz = ((cell >> 2) & 1) - 1 + X[k];
    const double w = W[i] * W[j] * W[k] * (1.0 - fabs(ox)) * (1.0 - fabs(oy)) * (1.0 - fabs(oz));
    const double v[3] = {dx + ox, dy + oy, dz + oz};
    const double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double r = sqrt(r2);
    double s, c;
    sincos(kappa * r, &s, &c);
    // d_a g = -(1 + j kappa r) e^{-j kappa r} v_a / (4 pi r^3)
    const double f = -w / (4.0 * M_PI * r * r2);
    const double kr = kappa * r;
    const double er = (c + kr * s) * f, ei = (kr * c - s) * f;   // (1 + j kr)(c - j s) f
    for (int a = 0; a < 3; ++a) {
      acc[2 * a] += er * v[a];
      acc[2 * a + 1] += ei * v[a];
    }
  }
  for (int k = 0; k < 6; ++k)
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  if (lane == 0)
    for (int a = 0; a < 3; ++a) C[a * N + gw] = make_double2(acc[2 * a], acc[2 * a + 1]);
}

// circulant embedding of C_a: odd along axis a, even along the others
__global__ void embed_curl_kernel(const double2* __restrict__ C, double2* __restrict__ full,
                                  int nx, int ny, int nz, int Mx, int My, int Mz) {
  const size_t total = (size_t)3 * Mx * My * Mz;
  const size_t N = (size_t)nx * ny * nz;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int mx = (int)(idx % Mx);
    const int my = (int)((idx / Mx) % My);
    const int mz = (int)((idx / ((size_t)Mx * My)) % Mz);
    const int a = (int)(idx / ((size_t)Mx * My * Mz));
    bool nx_, ny_, nz_, vx, vy, vz;
    const int dx = fold_index(mx, nx, Mx, &nx_, &vx);
    const int dy = fold_index(my, ny, My, &ny_, &vy);
    const int dz = fold_index(mz, nz, Mz, &nz_, &vz);
    double2 val = make_double2(0.0, 0.0);
    if (vx && vy && vz) {
      val = C[a * N + ((size_t)dz * ny + dy) * nx + dx];
      const bool flip = (a == 0) ? nx_ : (a == 1) ? ny_ : nz_;
      if (flip) { val.x = -val.x; val.y = -val.y; }
    }
    full[idx] = val;
  }
}

// fold to the octant [kx'][a][kz'][ky'], scaled by 1/(Mx My Mz)
__global__ void fold_curl_kernel(const double2* __restrict__ full, double2* __restrict__ c64,
                                 float2* __restrict__ c32, int Mx, int My, int Mz, int Kx, int Ky, int Kz,
                                 double scale_) {
  const size_t total = (size_t)Kx * 3 * Kz * Ky;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(idx % Ky);
    const int kz = (int)((idx / Ky) % Kz);
    const int a = (int)((idx / ((size_t)Ky * Kz)) % 3);
    const int kx = (int)(idx / ((size_t)Ky * Kz * 3));
    double2 v = full[(((size_t)a * Mz + kz) * My + ky) * Mx + kx];
    v.x *= scale_;
    v.y *= scale_;
    c64[idx] = v;
    c32[idx] = make_float2((float)v.x, (float)v.y);
  }
}

vie_status compute_curl(vie_plan* p, cudaStream_t s) {
  vie_status st = upload_gl_tables();
  if (st != VIE_OK) return st;
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int Mx = p->m[0], My = p->m[1], Mz = p->m[2];
  const size_t N = (size_t)nx * ny * nz;
  {
    const int threads = 256;
    const size_t blocks = (N * 32 + threads - 1) / threads;
    far_curl_kernel<<<(unsigned)blocks, threads, 0, s>>>(p->curl, nx, ny, nz, p->kappa);
    VIE_LAUNCH_CHECK();
    const size_t smem = (size_t)(threads / 32 + 1) * kNearAcc * 2 * sizeof(double);
    near_curl_kernel<<<8, threads, smem, s>>>(p->curl, nx, ny, nz, p->kappa);
    VIE_LAUNCH_CHECK();
  }
  const size_t cells = (size_t)Mx * My * Mz;
  double2* full = nullptr;
  VIE_CUDA_TRY(cudaMallocAsync((void**)&full, 3 * cells * sizeof(double2), s));
  {
    const size_t total = 3 * cells;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    embed_curl_kernel<<<blocks, 256, 0, s>>>(p->curl, full, nx, ny, nz, Mx, My, Mz);
    if (cudaGetLastError() != cudaSuccess) { set_error("embed_curl_kernel launch failed"); st = VIE_ERR_CUDA; }
  }
  if (st == VIE_OK) st = fft_axis_f64(full, p->ax[0], 1, 0, 3LL * Mz * My, Mx, 1, s);
  if (st == VIE_OK) st = fft_axis_f64(full, p->ax[1], 3LL * Mz, (long long)My * Mx, Mx, 1, Mx, s);
  if (st == VIE_OK) st = fft_axis_f64(full, p->ax[2], 3, (long long)Mz * My * Mx, (long long)My * Mx, 1,
                                      (long long)My * Mx, s);
  if (st == VIE_OK) {
    const size_t total = (size_t)p->kf[0] * 3 * p->kf[2] * p->kf[1];
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    fold_curl_kernel<<<blocks, 256, 0, s>>>(full, p->chat64, p->chat32, Mx, My, Mz, p->kf[0], p->kf[1], p->kf[2],
                                            1.0 / (double)cells);
    if (cudaGetLastError() != cudaSuccess) { set_error("fold_curl_kernel launch failed"); st = VIE_ERR_CUDA; }
  }
  cudaError_t e = cudaFreeAsync(full, s);
  if (st == VIE_OK && e != cudaSuccess) { set_error("cudaFreeAsync: %s", cudaGetErrorString(e)); st = VIE_ERR_CUDA; }
  return st;
}

}  // namespace vie
