// Block-circulant preconditioner of Sec. 5.4: the Frobenius-nearest matrix W
// to A = I - M N that is circulant in x, with dense (3 ny nz)^2 blocks.
//
// View A as nx x nx blocks A[i][j] (rows and columns ordered (p, z, y)):
// A[i][j] = delta_ij I - M_i T(i - j).  The nearest block-circulant matrix
// has the blocks c_k = (1/nx) sum_i A[i][(i - k) mod nx], i.e.
//   c_k = delta_k0 I - S+_k T(k) - S-_k T(k - nx),
//   S+_k = (1/nx) sum_{i >= k} M_i,  S-_k = (1/nx) sum_{i < k} M_i
// (row scalings by the x-averaged contrast).  The DFT along x
// block-diagonalises W: W_hat(w) = sum_k c_k exp(-2 pi i w k / nx).
//
// Setup (once per plan and contrast):
//   1. prefix sums of M along x (FP64),
//   2. W_hat: the blocks c_k of up to 16 entries at a time are formed in
//      shared memory and transformed along k by a Stockham FFT (radices 2-5
//      as butterflies, larger prime factors such as 7, 11, 13 summed
//      directly), so the blocks c_k are never stored,
//   3. LU with partial pivoting of the nx blocks W_hat(w): panels of nb
//      columns factored in shared memory, row swaps, a triangular solve for
//      the U row block, and the trailing update A22 -= L21 U12 as a batched
//      complex GEMM (64 x 64 output tiles per CTA, FP32).
// Application z = W^{-1} v (complex64):
//   V_hat = FFT along x of the 3 ny nz lines, one pivoted forward and
//   backward substitution per frequency (one CTA each, the factor streamed
//   once from HBM), then z = inverse FFT / nx.  The vectors' planar layout
//   [p][z][y][x] is already the (3B) x nx matrix the transforms need.
#include <cuda_fp16.h>
#include <math.h>
#include <stdio.h>

#include <chrono>

#include "fft.cuh"
#include "vie_internal.cuh"

struct vie_circulant {
  int device = 0;
  const vie_plan* plan = nullptr;
  int gen = 0;                 // contrast generation the factors were built from
  int nx = 0, ny = 0, nz = 0, B = 0, R = 0, nb = 32;
  float2* W = nullptr;         // nx x R x R: LU factors (unit L below, U on and above the diagonal)
  __half2* W16 = nullptr;      // the same in complex half precision (VIE_CIRC_FP16_FACTORS; W is then freed)
  bool fp16 = false;
  int* perm = nullptr;         // nx x R: row r of P b is b[perm[r]]
  float2* vh = nullptr;        // nx x R scratch (row-major [w][r])
  float2* v32 = nullptr;       // 3N scratch for complex128 callers
  float2* z32 = nullptr;
  int* flag = nullptr;         // 1: a zero pivot was met
  float2* tw = nullptr;        // nx twiddles exp(-2 pi i k / nx)
  vie::Radices rd;             //   and the radices of nx for the FFTs along x
  double build_ms = 0.0;
};

namespace vie {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 csub_mul(float2 acc, float2 a, float2 b) {
  // acc - a b
  return make_float2(acc.x - (a.x * b.x - a.y * b.y), acc.y - (a.x * b.y + a.y * b.x));
}

// ---------------------------------------------------------------------------
// setup kernels
// ---------------------------------------------------------------------------
// S+[zy][k] = (1/nx) sum_{i >= k} M[zy][i], S-[zy][k] = (1/nx) sum_{i < k} M[zy][i]
__global__ void prefix_kernel(const double2* __restrict__ M, int nx, int B, float2* __restrict__ Sp,
                              float2* __restrict__ Sm) {
  const int zy = blockIdx.x * blockDim.x + threadIdx.x;
  if (zy >= B) return;
  const double2* row = M + (size_t)zy * nx;
  double tx = 0.0, ty = 0.0;
  for (int i = 0; i < nx; ++i) {
    tx += row[i].x;
    ty += row[i].y;
  }
  double lx = 0.0, ly = 0.0;   // sum over i < k
  const double inv = 1.0 / nx;
  for (int k = 0; k < nx; ++k) {
    Sm[(size_t)zy * nx + k] = make_float2((float)(lx * inv), (float)(ly * inv));
    Sp[(size_t)zy * nx + k] = make_float2((float)((tx - lx) * inv), (float)((ty - ly) * inv));
    lx += row[k].x;
    ly += row[k].y;
  }
}

// Component index of (p, q) in the Toeplitz table order xx, yy, zz, xy, xz, yz.
__device__ __forceinline__ int comp_of(int p, int q) {
  if (p == q) return p;
  const int a = min(p, q), b = max(p, q);
  return a == 0 ? (b == 1 ? 3 : 4) : 5;
}

// T_pq(dx, dy, dz) for signed offsets from the octant table; an
// off-diagonal component is odd in each of its two axes.
__device__ __forceinline__ float2 toeplitz_at(const double2* __restrict__ T, int nx, int ny, int nz, int p, int q,
                                             int dx, int dy, int dz) {
  const int c = comp_of(p, q);
  const double2 t = T[(((size_t)c * nz + abs(dz)) * ny + abs(dy)) * nx + abs(dx)];
  float sgn = 1.f;
  if (p != q) {
    const int d[3] = {dx, dy, dz};
    if (d[p] < 0) sgn = -sgn;
    if (d[q] < 0) sgn = -sgn;
  }
  return make_float2(sgn * (float)t.x, sgn * (float)t.y);
}

// W_hat[w][e] for tl (<= kTL) consecutive entries e = r R + s at once:
// c_k[e] for every k is formed in shared memory and transformed along k by
// the Stockham FFT, so the blocks c_k are never stored.  tw = exp(-2 pi i k
// / nx).  tl is chosen so that the 2 tl lines of nx + 1 values fit in shared
// memory.
constexpr int kTL = 16;
__global__ void __launch_bounds__(256) build_fft_kernel(const double2* __restrict__ T, const float2* __restrict__ Sp,
                                                        const float2* __restrict__ Sm, int nx, int ny, int nz, int tl,
                                                        Radices rd, const float2* __restrict__ twg,
                                                        float2* __restrict__ What) {
  extern __shared__ float2 sb[];
  __shared__ const double2* tline[kTL];
  __shared__ float sgn_yz[kTL], sgn_neg[kTL];
  __shared__ int zyrow[kTL], diag[kTL];
  const int B = ny * nz, R = 3 * B;
  const long long RR = (long long)R * R;
  const int pitch = nx + 1;
  float2* tw = sb;
  float2* A = tw + nx;
  float2* Bf = A + tl * pitch;
  const long long e0 = (long long)blockIdx.x * tl;
  const int nl = (int)min((long long)tl, RR - e0);
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < nx; i += nth) tw[i] = twg[i];
  if (tid < nl) {
    const long long e = e0 + tid;
    const int r = (int)(e / R), s2 = (int)(e % R);
    const int p = r / B, zy = r % B, z = zy / ny, y = zy % ny;
    const int q = s2 / B, zy2 = s2 % B, z2 = zy2 / ny, y2 = zy2 % ny;
    const int dy = y - y2, dz = z - z2;
    const int c = comp_of(p, q);
    float sg = 1.f, sx = 1.f;
    if (p != q) {
      // odd in the axes of both components: y (1) and z (2) here, x (0) for the negative offsets k - nx
      if ((p == 1 || q == 1) && dy < 0) sg = -sg;
      if ((p == 2 || q == 2) && dz < 0) sg = -sg;
      if (p == 0 || q == 0) sx = -1.f;
    }
    tline[tid] = T + (((size_t)c * nz + abs(dz)) * ny + abs(dy)) * nx;
    sgn_yz[tid] = sg;
    sgn_neg[tid] = sg * sx;
    zyrow[tid] = zy;
    diag[tid] = (r == s2);
  }
  __syncthreads();
  for (int idx = tid; idx < nl * nx; idx += nth) {
    const int l = idx / nx, k = idx - l * nx;
    const double2* tl = tline[l];
    const double2 tp = tl[k];
    float2 out = make_float2((k == 0 && diag[l]) ? 1.f : 0.f, 0.f);
    const float2 sp = Sp[(size_t)zyrow[l] * nx + k];
    out = csub_mul(out, sp, make_float2(sgn_yz[l] * (float)tp.x, sgn_yz[l] * (float)tp.y));
    if (k > 0) {
      const double2 tn = tl[nx - k];
      const float2 sm = Sm[(size_t)zyrow[l] * nx + k];
      out = csub_mul(out, sm, make_float2(sgn_neg[l] * (float)tn.x, sgn_neg[l] * (float)tn.y));
    }
    A[l * pitch + k] = out;
  }
  for (int idx = nl * nx + tid; idx < tl * nx; idx += nth) A[(idx / nx) * pitch + idx % nx] = make_float2(0.f, 0.f);
  __syncthreads();
  const float2* res = fft_lines<float2, false, true>(A, Bf, rd, pitch, tl, tw, tid, nth);
  for (int idx = tid; idx < nx * tl; idx += nth) {
    const int w = idx / tl, l = idx - w * tl;
    if (l < nl) What[(size_t)w * RR + e0 + l] = res[l * pitch + w];
  }
}

__global__ void twiddle_kernel(int nx, float2* __restrict__ tw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nx) return;
  double sn, cs;
  sincospi(2.0 * (double)k / (double)nx, &sn, &cs);
  tw[k] = make_float2((float)cs, (float)-sn);
}

// DFTs along x of the application as FFTs, kLines rows per block.  Forward: vh[w][r] = sum_x v[r][x] exp(-2 pi i w x /
// nx); inverse: z[r][x] = (1/nx) sum_w vh[w][r] exp(+2 pi i w x / nx).
constexpr int kLines = 4;
template <bool INV>
__global__ void __launch_bounds__(256) lines_fft_kernel(const float2* __restrict__ in, float2* __restrict__ out, int R,
                                                        int nx, Radices rd, const float2* __restrict__ twg) {
  extern __shared__ float2 sb[];
  const int pitch = nx + 1;
  float2* tw = sb;
  float2* A = tw + nx;
  float2* Bf = A + kLines * pitch;
  const int r0 = blockIdx.x * kLines, nl = min(kLines, R - r0);
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < nx; i += nth) tw[i] = twg[i];
  for (int idx = tid; idx < kLines * nx; idx += nth) {
    int l, k;
    if (INV) { k = idx / kLines; l = idx - k * kLines; } else { l = idx / nx; k = idx - l * nx; }
    float2 v = make_float2(0.f, 0.f);
    if (l < nl) v = INV ? in[(size_t)k * R + r0 + l] : in[(size_t)(r0 + l) * nx + k];
    A[l * pitch + k] = v;
  }
  __syncthreads();
  const float2* res = fft_lines<float2, INV, true>(A, Bf, rd, pitch, kLines, tw, tid, nth);
  const float inv = 1.f / (float)nx;
  for (int idx = tid; idx < kLines * nx; idx += nth) {
    int l, k;
    if (INV) { l = idx / nx; k = idx - l * nx; } else { k = idx / kLines; l = idx - k * kLines; }
    if (l >= nl) continue;
    const float2 v = res[l * pitch + k];
    if (INV) out[(size_t)(r0 + l) * nx + k] = make_float2(v.x * inv, v.y * inv);
    else out[(size_t)k * R + r0 + l] = v;
  }
}

// ---------------------------------------------------------------------------
// batched LU with partial pivoting (row-major blocks, one matrix per CTA)
// ---------------------------------------------------------------------------
// Panel j0 .. j0 + nbe - 1 of every matrix, rows j0 .. R - 1, factored in
// shared memory (pitch nbe + 1): per column the largest |a| below the
// diagonal is the pivot (lowest row on ties), rows are swapped inside the
// panel, the column is scaled by the pivot's inverse and the rest of the
// panel gets the rank-1 update.  piv[j] = the row swapped with row j.
__global__ void __launch_bounds__(256) lu_panel_kernel(float2* __restrict__ W, int R, int j0, int nbe,
                                                       int* __restrict__ piv, int* __restrict__ flag) {
  extern __shared__ float2 P[];
  __shared__ float bval[8];
  __shared__ int bidx[8];
  __shared__ int ipiv;
  float2* A = W + (size_t)blockIdx.x * R * R;
  const int rows = R - j0, pitch = nbe + 1;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < rows * nbe; e += nth) {
    const int i = e / nbe, c = e - i * nbe;
    P[i * pitch + c] = A[(size_t)(j0 + i) * R + j0 + c];
  }
  __syncthreads();
  for (int jj = 0; jj < nbe; ++jj) {
    // pivot search over rows jj .. rows - 1 of column jj
    float best = -1.f;
    int bi = rows;
    for (int i = jj + tid; i < rows; i += nth) {
      const float2 a = P[i * pitch + jj];
      const float m = a.x * a.x + a.y * a.y;
      if (m > best) { best = m; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { bval[wid] = best; bidx[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      float b = bval[0];
      int ii = bidx[0];
      for (int w = 1; w < (nth >> 5); ++w)
        if (bval[w] > b || (bval[w] == b && bidx[w] < ii)) { b = bval[w]; ii = bidx[w]; }
      if (!(b > 0.f)) { atomicExch(flag, 1); ii = jj; }
      ipiv = ii;
      piv[(size_t)blockIdx.x * R + j0 + jj] = j0 + ii;
    }
    __syncthreads();
    const int ip = ipiv;
    if (ip != jj)
      for (int c = tid; c < nbe; c += nth) {
        const float2 t = P[jj * pitch + c];
        P[jj * pitch + c] = P[ip * pitch + c];
        P[ip * pitch + c] = t;
      }
    __syncthreads();
    const float2 d = P[jj * pitch + jj];
    const float dd = d.x * d.x + d.y * d.y;
    const float2 inv = dd > 0.f ? make_float2(d.x / dd, -d.y / dd) : make_float2(0.f, 0.f);
    for (int i = jj + 1 + tid; i < rows; i += nth) {
      const float2 l = cmul(P[i * pitch + jj], inv);
      P[i * pitch + jj] = l;
      for (int c = jj + 1; c < nbe; ++c) P[i * pitch + c] = csub_mul(P[i * pitch + c], l, P[jj * pitch + c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < rows * nbe; e += nth) {
    const int i = e / nbe, c = e - i * nbe;
    A[(size_t)(j0 + i) * R + j0 + c] = P[i * pitch + c];
  }
}

// The panel's row swaps applied to every column outside it (the L columns
// to its left included, as in the usual packed LU).  One thread per column.
__global__ void __launch_bounds__(256) lu_swap_kernel(float2* __restrict__ W, int R, int j0, int nbe,
                                                      const int* __restrict__ piv) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= R || (c >= j0 && c < j0 + nbe)) return;
  float2* A = W + (size_t)blockIdx.x * R * R;
  const int* pv = piv + (size_t)blockIdx.x * R;
  for (int jj = 0; jj < nbe; ++jj) {
    const int r1 = j0 + jj, r2 = pv[r1];
    if (r2 != r1) {
      const float2 t = A[(size_t)r1 * R + c];
      A[(size_t)r1 * R + c] = A[(size_t)r2 * R + c];
      A[(size_t)r2 * R + c] = t;
    }
  }
}

// U12 = L11^{-1} A12: rows j0 .. j0 + NB - 1, columns j0 + NB .. R - 1; L11
// is the unit lower triangle of the factored panel.  One thread per column.
template <int NB>
__global__ void __launch_bounds__(256) lu_trsm_kernel(float2* __restrict__ W, int R, int j0) {
  __shared__ float2 L[NB][NB + 1];
  float2* A = W + (size_t)blockIdx.x * R * R;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, t = e - i * NB;
    L[i][t] = A[(size_t)(j0 + i) * R + j0 + t];
  }
  __syncthreads();
  const int c = j0 + NB + blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= R) return;
  float2 x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) x[i] = A[(size_t)(j0 + i) * R + c];
#pragma unroll
  for (int i = 1; i < NB; ++i)
#pragma unroll
    for (int t = 0; t < i; ++t) x[i] = csub_mul(x[i], L[i][t], x[t]);
#pragma unroll
  for (int i = 0; i < NB; ++i) A[(size_t)(j0 + i) * R + c] = x[i];
}

// Trailing update A22 -= L21 U12 of every matrix (blockIdx.z): L21 = rows
// j1 .. R - 1, columns j0 .. j1 - 1; U12 = rows j0 .. j1 - 1, columns
// j1 .. R - 1 (KB = j1 - j0).  One CTA per 64 x 64 tile of A22: the two
// operand panels are staged in shared memory (L21 transposed), each of the
// 256 threads accumulates 4 x 4 complex products (rows ty + 16 a, columns
// tx + 16 b, so that a warp's stores cover 16 consecutive columns).  The
// regions read and written are disjoint, so the update is in place.
template <int KB>
__global__ void __launch_bounds__(256) lu_update_kernel(float2* __restrict__ W, int R, int j0) {
  __shared__ float2 As[KB][65];
  __shared__ float2 Bs[KB][64];
  float2* A = W + (size_t)blockIdx.z * R * R;
  const int j1 = j0 + KB, n = R - j1;
  const int i0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const int tid = threadIdx.x;
  for (int e = tid; e < 64 * KB; e += 256) {
    const int i = e / KB, k = e - i * KB;
    const int r = i0 + i;
    As[k][i] = r < n ? A[(size_t)(j1 + r) * R + j0 + k] : make_float2(0.f, 0.f);
  }
  for (int e = tid; e < 64 * KB; e += 256) {
    const int k = e >> 6, j = e & 63;
    const int c = c0 + j;
    Bs[k][j] = c < n ? A[(size_t)(j0 + k) * R + j1 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int k = 0; k < KB; ++k) {
    float2 av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        acc[a][b].x = fmaf(av[a].x, bv[b].x, fmaf(-av[a].y, bv[b].y, acc[a][b].x));
        acc[a][b].y = fmaf(av[a].x, bv[b].y, fmaf(av[a].y, bv[b].x, acc[a][b].y));
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = i0 + ty + 16 * a;
    if (r >= n) continue;
    float2* row = A + (size_t)(j1 + r) * R + j1;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx + 16 * b;
      if (c < n) {
        float2 v = row[c];
        v.x -= acc[a][b].x;
        v.y -= acc[a][b].y;
        row[c] = v;
      }
    }
  }
}

// perm[w][r]: the swaps piv[w][0 .. R) applied in order to the identity, so
// that (P b)[r] = b[perm[r]].  One thread per matrix.
__global__ void perm_kernel(const int* __restrict__ piv, int R, int nmat, int* __restrict__ perm) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nmat) return;
  int* pm = perm + (size_t)w * R;
  const int* pv = piv + (size_t)w * R;
  for (int r = 0; r < R; ++r) pm[r] = r;
  for (int r = 0; r < R; ++r) {
    const int o = pv[r];
    if (o != r) {
      const int t = pm[r];
      pm[r] = pm[o];
      pm[o] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// application: one CTA per frequency solves W_hat(w) z = b in place
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  const float d = b.x * b.x + b.y * b.y;
  return make_float2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ __forceinline__ float2 ld_factor(const float2* p) { return *p; }
__device__ __forceinline__ float2 ld_factor(const __half2* p) { return __half22float2(*p); }

// Streamer part of the pipelined substitution: 224 threads (warps 1-7),
// seven per row of a 32-row block row.  Thread (row, sub) sums
// A[j0 + row][t] x[t] over t = c0 + sub + 7 u < c1 with 16 (complex64) or 32
// (complex half) loads in flight and leaves the sum in red[row][sub].
template <typename T>
__device__ __forceinline__ void stream_partial(const T* __restrict__ A, int R, int j0, int nr, int c0, int c1,
                                               const float2* __restrict__ x, float2 (*red)[8], int st) {
  const int row = st / 7, sub = st - row * 7;
  float sx = 0.f, sy = 0.f;
  if (row < nr) {
    constexpr int U = sizeof(T) == 4 ? 32 : 16;
    const T* rp = A + (size_t)(j0 + row) * R;
    int t = c0 + sub;
    for (; t + 7 * (U - 1) < c1; t += 7 * U) {
      float2 l[U];
#pragma unroll
      for (int u = 0; u < U; ++u) l[u] = ld_factor(rp + t + 7 * u);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float2 xt = x[t + 7 * u];
        sx += l[u].x * xt.x - l[u].y * xt.y;
        sy += l[u].x * xt.y + l[u].y * xt.x;
      }
    }
    for (; t < c1; t += 7) {
      const float2 l = ld_factor(rp + t), xt = x[t];
      sx += l.x * xt.x - l.y * xt.y;
      sy += l.x * xt.y + l.y * xt.x;
    }
  }
  red[row][sub] = make_float2(sx, sy);
}

// x = P b (gather), then L y = x and U z = y in blocks of 32 rows, pipelined:
// while warp 0 solves block k (its rows minus the streamed partial and the
// coupling to the block solved just before, then the 32 x 32 diagonal block
// with shuffles), warps 1-7 stream block k+1's products with every column
// that is already final and prefetch block k+1's diagonal block and its
// coupling block into the other half of double-buffered shared memory.  One
// barrier per block.  256 threads.
template <typename T>
__global__ void __launch_bounds__(256, 4) circ_solve_kernel(const T* __restrict__ W, const int* __restrict__ perm,
                                                         float2* __restrict__ vh, int R) {
  extern __shared__ float2 x[];
  __shared__ float2 D[2][32][33];   // diagonal block
  __shared__ float2 E[2][32][33];   // coupling to the previously solved block
  __shared__ float2 red[2][32][8];  // streamed partial sums, 7 per row
  const T* A = W + (size_t)blockIdx.x * R * R;
  const int* pm = perm + (size_t)blockIdx.x * R;
  float2* b = vh + (size_t)blockIdx.x * R;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, st = tid - 32;
  const int nblk = (R + 31) / 32;
  auto nrows = [&](int k) { return min(32, R - 32 * k); };
  for (int r = tid; r < R; r += blockDim.x) x[r] = b[pm[r]];
  // ---------------- forward: unit lower L ----------------
  {
    const int nr = nrows(0);
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int a = e >> 5, t = e & 31;
      D[0][a][t] = (a < nr && t < nr) ? ld_factor(A + (size_t)a * R + t) : make_float2(0.f, 0.f);
      if (t < 8) red[0][a][t] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  for (int k = 0; k < nblk; ++k) {
    const int cur = k & 1, nxt = cur ^ 1, i0 = 32 * k, nr = nrows(k);
    if (wid == 0) {
      float2 xi = lane < nr ? x[i0 + lane] : make_float2(0.f, 0.f);
      if (lane < nr) {
#pragma unroll
        for (int q = 0; q < 7; ++q) xi = make_float2(xi.x - red[cur][lane][q].x, xi.y - red[cur][lane][q].y);
        if (k > 0)
          for (int t = 0; t < 32; ++t) xi = csub_mul(xi, E[cur][lane][t], x[i0 - 32 + t]);
      }
      for (int t = 0; t < nr; ++t) {
        const float2 xt = make_float2(__shfl_sync(0xffffffffu, xi.x, t), __shfl_sync(0xffffffffu, xi.y, t));
        if (lane > t && lane < nr) xi = csub_mul(xi, D[cur][lane][t], xt);
      }
      if (lane < nr) x[i0 + lane] = xi;
    } else if (k + 1 < nblk) {
      const int j0 = i0 + 32, nr1 = nrows(k + 1);
      stream_partial(A, R, j0, nr1, 0, i0, x, red[nxt], st);
      for (int e = st; e < 32 * 32; e += blockDim.x - 32) {
        const int a = e >> 5, t = e & 31;
        const bool in = a < nr1;
        D[nxt][a][t] = (in && t < nr1) ? ld_factor(A + (size_t)(j0 + a) * R + j0 + t) : make_float2(0.f, 0.f);
        E[nxt][a][t] = in ? ld_factor(A + (size_t)(j0 + a) * R + i0 + t) : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
  }
  // ---------------- backward: upper U with its diagonal ----------------
  {
    const int kl = nblk - 1, i0 = 32 * kl, nr = nrows(kl);
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int a = e >> 5, t = e & 31;
      D[0][a][t] = (a < nr && t < nr) ? ld_factor(A + (size_t)(i0 + a) * R + i0 + t) : make_float2(0.f, 0.f);
      if (t < 8) red[0][a][t] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  for (int it = 0; it < nblk; ++it) {
    const int k = nblk - 1 - it, cur = it & 1, nxt = cur ^ 1;
    const int i0 = 32 * k, nr = nrows(k), i1 = i0 + nr;
    if (wid == 0) {
      float2 xi = lane < nr ? x[i0 + lane] : make_float2(0.f, 0.f);
      if (lane < nr) {
#pragma unroll
        for (int q = 0; q < 7; ++q) xi = make_float2(xi.x - red[cur][lane][q].x, xi.y - red[cur][lane][q].y);
        if (k + 1 < nblk) {
          const int nrn = nrows(k + 1);
          for (int t = 0; t < nrn; ++t) xi = csub_mul(xi, E[cur][lane][t], x[i1 + t]);
        }
      }
      for (int t = nr - 1; t >= 0; --t) {
        if (lane == t) xi = cdiv(xi, D[cur][t][t]);
        const float2 xt = make_float2(__shfl_sync(0xffffffffu, xi.x, t), __shfl_sync(0xffffffffu, xi.y, t));
        if (lane < t) xi = csub_mul(xi, D[cur][lane][t], xt);
      }
      if (lane < nr) x[i0 + lane] = xi;
    } else if (k > 0) {
      const int j0 = i0 - 32;      // block k - 1 has 32 rows
      stream_partial(A, R, j0, 32, i1, R, x, red[nxt], st);
      for (int e = st; e < 32 * 32; e += blockDim.x - 32) {
        const int a = e >> 5, t = e & 31;
        D[nxt][a][t] = ld_factor(A + (size_t)(j0 + a) * R + j0 + t);
        E[nxt][a][t] = t < nr ? ld_factor(A + (size_t)(j0 + a) * R + i0 + t) : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
  }
  for (int r = tid; r < R; r += blockDim.x) b[r] = x[r];
}

__global__ void to_half_kernel(const float2* __restrict__ a, __half2* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = __float22half2_rn(a[i]);
}

__global__ void to_c64_kernel(const double2* __restrict__ a, float2* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void to_c128_kernel(const float2* __restrict__ a, double2* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

static unsigned blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static void circ_free(vie_circulant* c) {
  if (!c) return;
  cudaFree(c->W); cudaFree(c->W16); cudaFree(c->tw); cudaFree(c->perm); cudaFree(c->vh);
  cudaFree(c->v32); cudaFree(c->z32); cudaFree(c->flag);
  delete c;
}

// Lines per block of the fused build (blocks formed and transformed along x
// in shared memory): the largest of 16, 8, 4, 2, 1 whose two buffers of
// nx + 1 values and the twiddle table fit in `smem_max` bytes, or 0.
static int build_lines(int nx, size_t smem_max) {
  for (int tl = kTL; tl >= 1; tl >>= 1)
    if ((size_t)nx * sizeof(float2) + (size_t)2 * tl * (nx + 1) * sizeof(float2) <= smem_max) return tl;
  return 0;
}

static vie_status circ_build(vie_circulant* c, cudaStream_t s, size_t smem_max) {
  const vie_plan* p = c->plan;
  const int nx = c->nx, ny = c->ny, nz = c->nz, B = c->B, R = c->R;
  const size_t RR = (size_t)R * R, N3 = (size_t)3 * B * nx;
  float2 *Sp = nullptr, *Sm = nullptr;
  int* piv = nullptr;
  vie_status st = VIE_OK;
  auto fail = [&](vie_status e) { cudaFree(Sp); cudaFree(Sm); cudaFree(piv); return e; };
#define CIRC_TRY(expr)                                                                         \
  do {                                                                                         \
    cudaError_t e__ = (expr);                                                                  \
    if (e__ != cudaSuccess) {                                                                  \
      set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e__));   \
      return fail(e__ == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA);             \
    }                                                                                          \
  } while (0)
  CIRC_TRY(cudaMalloc((void**)&Sp, (size_t)nx * B * sizeof(float2)));
  CIRC_TRY(cudaMalloc((void**)&Sm, (size_t)nx * B * sizeof(float2)));
  CIRC_TRY(cudaMalloc((void**)&piv, (size_t)nx * R * sizeof(int)));
  CIRC_TRY(cudaMalloc((void**)&c->W, (size_t)nx * RR * sizeof(float2)));
  CIRC_TRY(cudaMalloc((void**)&c->perm, (size_t)nx * R * sizeof(int)));
  CIRC_TRY(cudaMalloc((void**)&c->vh, (size_t)nx * R * sizeof(float2)));
  CIRC_TRY(cudaMalloc((void**)&c->v32, N3 * sizeof(float2)));
  CIRC_TRY(cudaMalloc((void**)&c->z32, N3 * sizeof(float2)));
  CIRC_TRY(cudaMalloc((void**)&c->flag, sizeof(int)));
  CIRC_TRY(cudaMalloc((void**)&c->tw, (size_t)nx * sizeof(float2)));
  CIRC_TRY(cudaMemsetAsync(c->flag, 0, sizeof(int), s));

  prefix_kernel<<<(B + 127) / 128, 128, 0, s>>>(p->M64, nx, B, Sp, Sm);
  twiddle_kernel<<<(nx + 127) / 128, 128, 0, s>>>(nx, c->tw);
  CIRC_TRY(cudaGetLastError());
  // W_hat: blocks formed and transformed along x in shared memory
  const int tl = build_lines(nx, smem_max);
  const size_t fft_smem = (size_t)nx * sizeof(float2) + (size_t)2 * tl * (nx + 1) * sizeof(float2);
  CIRC_TRY(cudaFuncSetAttribute(build_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem));
  build_fft_kernel<<<(unsigned)((RR + tl - 1) / tl), 256, fft_smem, s>>>(p->toeplitz, Sp, Sm, nx, ny, nz, tl, c->rd,
                                                                        c->tw, c->W);
  CIRC_TRY(cudaGetLastError());
  // LU of the nx blocks
  const int nb = c->nb;
  for (int j0 = 0; j0 < R; j0 += nb) {
    const int nbe = min(nb, R - j0), j1 = j0 + nbe;
    const size_t smem = (size_t)(R - j0) * (nbe + 1) * sizeof(float2);
    CIRC_TRY(cudaFuncSetAttribute(lu_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    lu_panel_kernel<<<nx, 256, smem, s>>>(c->W, R, j0, nbe, piv, c->flag);
    lu_swap_kernel<<<dim3(nx, (R + 255) / 256), 256, 0, s>>>(c->W, R, j0, nbe, piv);
    CIRC_TRY(cudaGetLastError());
    if (j1 < R) {
      // here nbe == nb: only the last panel can be narrower, and it has no trailing block
      const dim3 tg(nx, (R - j1 + 255) / 256);
      const unsigned tiles = (unsigned)((R - j1 + 63) / 64);
      if (nb == 32) {
        lu_trsm_kernel<32><<<tg, 256, 0, s>>>(c->W, R, j0);
        lu_update_kernel<32><<<dim3(tiles, tiles, nx), 256, 0, s>>>(c->W, R, j0);
      } else {
        lu_trsm_kernel<16><<<tg, 256, 0, s>>>(c->W, R, j0);
        lu_update_kernel<16><<<dim3(tiles, tiles, nx), 256, 0, s>>>(c->W, R, j0);
      }
      CIRC_TRY(cudaGetLastError());
    }
  }
  perm_kernel<<<(nx + 127) / 128, 128, 0, s>>>(piv, R, nx, c->perm);
  CIRC_TRY(cudaGetLastError());
  CIRC_TRY(cudaStreamSynchronize(s));
  int flag = 0;
  CIRC_TRY(cudaMemcpy(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost));
  fail(VIE_OK);
  Sp = Sm = nullptr;
  piv = nullptr;
  if (flag) {
    set_error("block-circulant preconditioner: a diagonal block is singular");
    st = VIE_ERR_NONFINITE;
  }
#undef CIRC_TRY
  return st;
}

const vie_plan* circulant_plan(const vie_circulant* c) { return c->plan; }

vie_status circulant_apply(vie_circulant* c, int dtype, const void* v, void* z, cudaStream_t s) {
  if (c->gen != c->plan->contrast_gen) {
    set_error("block-circulant preconditioner is stale: the plan's contrast changed after it was built");
    return VIE_ERR_INVALID;
  }
  const int nx = c->nx, R = c->R;
  const size_t N3 = (size_t)R * nx;
  const float2* vin = (const float2*)v;
  float2* zout = (float2*)z;
  if (dtype == VIE_C128) {
    to_c64_kernel<<<blocks_for(N3), 256, 0, s>>>((const double2*)v, c->v32, N3);
    VIE_LAUNCH_CHECK();
    vin = c->v32;
    zout = c->z32;
  }
  const size_t fft_smem = (size_t)nx * sizeof(float2) + (size_t)2 * kLines * (nx + 1) * sizeof(float2);
  VIE_CUDA_TRY(cudaFuncSetAttribute(lines_fft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem));
  VIE_CUDA_TRY(cudaFuncSetAttribute(lines_fft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem));
  // V_hat[w][r] = sum_x exp(-2 pi i w x / nx) v[r][x]
  lines_fft_kernel<false><<<(R + kLines - 1) / kLines, 256, fft_smem, s>>>(vin, c->vh, R, nx, c->rd, c->tw);
  VIE_LAUNCH_CHECK();
  if (c->fp16) circ_solve_kernel<__half2><<<nx, 256, (size_t)R * sizeof(float2), s>>>(c->W16, c->perm, c->vh, R);
  else circ_solve_kernel<float2><<<nx, 256, (size_t)R * sizeof(float2), s>>>(c->W, c->perm, c->vh, R);
  VIE_LAUNCH_CHECK();
  // z[r][x] = (1/nx) sum_w exp(+2 pi i w x / nx) Z_hat[w][r]
  lines_fft_kernel<true><<<(R + kLines - 1) / kLines, 256, fft_smem, s>>>(c->vh, zout, R, nx, c->rd, c->tw);
  VIE_LAUNCH_CHECK();
  if (dtype == VIE_C128) {
    to_c128_kernel<<<blocks_for(N3), 256, 0, s>>>(c->z32, (double2*)z, N3);
    VIE_LAUNCH_CHECK();
  }
  return VIE_OK;
}

}  // namespace vie

using namespace vie;

extern "C" {

vie_status vie_circulant_create(vie_plan* plan, int flags, vie_circulant** out, void* stream) {
  clear_error();
  if (!plan || !out) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (flags & ~VIE_CIRC_FP16_FACTORS) { set_error("unknown flags 0x%x", flags); return VIE_ERR_INVALID; }
  *out = nullptr;
  if (!plan->M64) { set_error("set the plan's contrast before building its circulant preconditioner"); return VIE_ERR_INVALID; }
  const auto t0 = std::chrono::steady_clock::now();
  vie_circulant* c = new vie_circulant();
  c->plan = plan;
  c->gen = plan->contrast_gen;
  c->nx = plan->n[0];
  c->ny = plan->n[1];
  c->nz = plan->n[2];
  c->B = c->ny * c->nz;
  c->R = 3 * c->B;
  // the panel (R rows x nb columns) must fit in shared memory
  const size_t budget = 220 * 1024;
  c->nb = (size_t)c->R * 33 * sizeof(float2) <= budget ? 32 : 16;
  if ((size_t)c->R * 17 * sizeof(float2) > budget) {
    set_error("cross-section of %d unknowns is too large for the block-circulant preconditioner", c->R);
    delete c;
    return VIE_ERR_INVALID;
  }
  if ((size_t)c->R * c->R > (size_t)0x7fffffff) {
    set_error("cross-section too large for the block-circulant preconditioner");
    delete c;
    return VIE_ERR_INVALID;
  }
  VIE_CUDA_TRY(cudaGetDevice(&c->device));
  int smem_optin = 0;
  VIE_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  // the FFTs along x: radices of nx (any prime factors) and shared memory for
  // the application's kLines lines and at least one line of the build
  AxisPlan ax;
  if (!factor_length_any(c->nx, &ax) ||
      (size_t)c->nx * sizeof(float2) + (size_t)2 * kLines * (c->nx + 1) * sizeof(float2) > (size_t)smem_optin ||
      build_lines(c->nx, (size_t)smem_optin) == 0) {
    set_error("nx = %d is too long for the block-circulant preconditioner's FFTs along x", c->nx);
    delete c;
    return VIE_ERR_INVALID;
  }
  c->rd = radices_of(ax);
  vie_status st = circ_build(c, (cudaStream_t)stream, (size_t)smem_optin);
  if (st == VIE_OK && (flags & VIE_CIRC_FP16_FACTORS)) {
    // keep only a complex-half copy of the factors
    const size_t ne = (size_t)c->nx * c->R * c->R;
    cudaError_t e = cudaMalloc((void**)&c->W16, ne * sizeof(__half2));
    if (e == cudaSuccess) {
      to_half_kernel<<<blocks_for(ne), 256, 0, (cudaStream_t)stream>>>(c->W, c->W16, ne);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
      set_error("half-precision factors: %s", cudaGetErrorString(e));
      st = e == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA;
    } else {
      cudaFree(c->W);
      c->W = nullptr;
      c->fp16 = true;
    }
  }
  if (st != VIE_OK) {
    circ_free(c);
    return st;
  }
  c->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = c;
  return VIE_OK;
}

vie_status vie_circulant_apply(vie_circulant* c, const void* v_dev, void* z_dev, int dtype, void* stream) {
  clear_error();
  if (!c || !v_dev || !z_dev) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (dtype != VIE_C64 && dtype != VIE_C128) { set_error("dtype must be VIE_C64 or VIE_C128"); return VIE_ERR_INVALID; }
  return circulant_apply(c, dtype, v_dev, z_dev, (cudaStream_t)stream);
}

vie_status vie_circulant_info(const vie_circulant* c, double* build_ms, size_t* device_bytes) {
  clear_error();
  if (!c) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (build_ms) *build_ms = c->build_ms;
  if (device_bytes)
    *device_bytes = (size_t)c->nx * c->R * c->R * (c->fp16 ? sizeof(__half2) : sizeof(float2)) +
                    (size_t)c->nx * c->R * (sizeof(int) + sizeof(float2)) + (size_t)c->nx * sizeof(float2) +
                    (size_t)2 * c->nx * c->R * sizeof(float2);
  return VIE_OK;
}

vie_status vie_circulant_destroy(vie_circulant* c) {
  circ_free(c);
  return VIE_OK;
}

}  // extern "C"
