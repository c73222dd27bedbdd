// Learned right preconditioner z = Net(v, chi): a 3-D convolutional network
// trained on the device by the kernels in this file.
//
// The paper preconditions GMRES with a block-circulant matrix (Sec. 5.4); the
// network is this project's addition.  Architecture (same as the oracle's):
// 8 input channels (re/im of the three components of v, re/im of chi), four
// levels (average pooling 2 x 2 in x and y, z kept), 32 channels, 3x3x3 convs
// with zero padding and bias, ReLU, nearest upsampling with additive skips,
// 6 output channels (re/im of the three components of z).  Weights are kept
// in FP32 for the optimiser and used as BF16 by the convolutions, which
// accumulate in FP32.  Training (this file) keeps FP32 planar activations;
// inference (conv_tc.cu) runs the convolutions on the tcgen05 tensor cores
// with channels-last BF16 activations.
//
// The preconditioner is z = v + Net(v): the network learns the correction
// to the identity, and its output layer starts at zero, so an untrained
// network is exactly the identity.  It is positively homogeneous: v is scaled
// to unit RMS before the network and the output is scaled back, so
// P(a v) = a P(v) for a > 0.  A non-finite output is replaced by v and
// reported.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "net.cuh"
#include "vie_internal.cuh"

namespace vie { struct TcCache; struct TcTrain; }

struct vie_net {
  int device = 0;
  size_t nparams = 0;
  float* master = nullptr;        // FP32 parameters: per layer w[co][ci][27] then b[co]
  float* grad = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  __nv_bfloat16* wbf = nullptr;   // BF16 copy of the parameters (same offsets)
  __nv_bfloat16* wflip = nullptr; // per layer w'[c][o][26 - t] (backward data)
  __nv_bfloat16* wpack = nullptr; // per layer tensor-core layout wp[tap][o][c] (inference)
  __nv_bfloat16* wpackf = nullptr;// per layer flipped weights in that layout (tensor-core backward data)
  vie::TcCache* tc = nullptr;     // inference workspace and tensor maps
  vie::TcTrain* train = nullptr;  // tensor-core training workspace and tensor maps
  int train_mode = VIE_TRAIN_TENSOR_BF16;
  long step = 0;
  float* ws = nullptr;            // activation workspace
  size_t ws_cap = 0;
  float* partial = nullptr;       // weight-gradient partial sums
  size_t partial_cap = 0;
  float* scal = nullptr;          // device scalars (norms, loss)
  int* bad = nullptr;             // non-finite output seen
};

namespace vie {

// ---------------------------------------------------------------------------
// convolution (forward; also the backward-data pass with flipped weights)
// Block: 128 threads on one (z, y) row, each thread 4 consecutive x.
// Weights of 16 input channels at a time in shared memory, [c][t][o].
// ---------------------------------------------------------------------------
constexpr int kConvThreads = 128;
constexpr int kConvVox = 4;
constexpr int kConvCiChunk = 16;

template <int CO>
__global__ void __launch_bounds__(kConvThreads) conv_fwd_kernel(const float* __restrict__ in, int ci,
                                                                const __nv_bfloat16* __restrict__ w,
                                                                const float* __restrict__ bias,
                                                                float* __restrict__ pre, float* __restrict__ out,
                                                                Dims d, int relu) {
  __shared__ float ws[kConvCiChunk * 27 * CO];
  const int z = blockIdx.z, y = blockIdx.y;
  const int xb = (blockIdx.x * kConvThreads + threadIdx.x) * kConvVox;
  const size_t plane = (size_t)d.ny * d.nx;
  const size_t chan = (size_t)d.nz * plane;
  float acc[kConvVox][CO];
#pragma unroll
  for (int v = 0; v < kConvVox; ++v)
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[v][o] = 0.f;
  for (int c0 = 0; c0 < ci; c0 += kConvCiChunk) {
    const int cn = min(kConvCiChunk, ci - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cn * 27 * CO; i += blockDim.x) {
      const int o = i % CO, t = (i / CO) % 27, c = i / (CO * 27);
      ws[i] = __bfloat162float(w[((size_t)o * ci + c0 + c) * 27 + t]);
    }
    __syncthreads();
    for (int c = 0; c < cn; ++c) {
      const float* inc = in + (size_t)(c0 + c) * chan;
      for (int dz = 0; dz < 3; ++dz) {
        const int zz = z + dz - 1;
        if (zz < 0 || zz >= d.nz) continue;
        for (int dy = 0; dy < 3; ++dy) {
          const int yy = y + dy - 1;
          if (yy < 0 || yy >= d.ny) continue;
          const float* row = inc + (size_t)zz * plane + (size_t)yy * d.nx;
          float xs[kConvVox + 2];
#pragma unroll
          for (int k = 0; k < kConvVox + 2; ++k) {
            const int xx = xb + k - 1;
            xs[k] = (xx >= 0 && xx < d.nx) ? row[xx] : 0.f;
          }
          const float* wt = ws + (c * 27 + dz * 9 + dy * 3) * CO;
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
            for (int o = 0; o < CO; ++o) {
              const float wv = wt[dx * CO + o];
#pragma unroll
              for (int v = 0; v < kConvVox; ++v) acc[v][o] = fmaf(wv, xs[v + dx], acc[v][o]);
            }
          }
        }
      }
    }
  }
  const size_t base = (size_t)z * plane + (size_t)y * d.nx;
#pragma unroll
  for (int v = 0; v < kConvVox; ++v) {
    const int x = xb + v;
    if (x >= d.nx) continue;
#pragma unroll
    for (int o = 0; o < CO; ++o) {
      const float val = acc[v][o] + (bias ? bias[o] : 0.f);
      if (pre) pre[(size_t)o * chan + base + x] = val;
      out[(size_t)o * chan + base + x] = relu ? fmaxf(val, 0.f) : val;
    }
  }
}

// wp[tap][o][c] (o < no, c < cip) from w[o][c][tap] (BF16), zero padding: the
// tensor-core layout, K-major rows of cip channels for each output channel
__global__ void pack_mma_weights_kernel(const __nv_bfloat16* __restrict__ w, int ci, int co, int cip, int no,
                                        __nv_bfloat16* __restrict__ wp) {
  const size_t n = (size_t)27 * no * cip;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % cip);
    const int o = (int)((i / cip) % no);
    const int t = (int)(i / ((size_t)cip * no));
    wp[i] = (o < co && c < ci) ? w[((size_t)o * ci + c) * 27 + t] : __float2bfloat16_rn(0.f);
  }
}

// dW[o][c][t] partial sums over the rows of one block, and the rows it owns:
// rows r = blockIdx.y, blockIdx.y + gridDim.y, ...; 8 input channels per block
// (blockIdx.x), thread = (o, c in chunk).  partial[(blockIdx.y * ci + c) * co + o][27]
__global__ void __launch_bounds__(256) conv_dw_kernel(const float* __restrict__ in, int ci,
                                                      const float* __restrict__ dout, int co, Dims d,
                                                      float* __restrict__ partial) {
  constexpr int XT = 64;
  __shared__ float sd[32][XT];
  __shared__ float si[8][9][XT + 2];
  const int c0 = blockIdx.x * 8;
  const int tid = threadIdx.x;
  const int o = tid / 8, cl = tid % 8;
  const bool active = (o < co) && (c0 + cl < ci);
  const size_t plane = (size_t)d.ny * d.nx;
  const size_t chan = (size_t)d.nz * plane;
  float acc[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) acc[t] = 0.f;
  const int rows = d.nz * d.ny;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int z = r / d.ny, y = r - z * d.ny;
    for (int x0 = 0; x0 < d.nx; x0 += XT) {
      __syncthreads();
      for (int i = tid; i < 32 * XT; i += blockDim.x) {
        const int oo = i / XT, xx = x0 + (i % XT);
        sd[oo][i % XT] = (oo < co && xx < d.nx) ? dout[(size_t)oo * chan + (size_t)z * plane + (size_t)y * d.nx + xx] : 0.f;
      }
      for (int i = tid; i < 8 * 9 * (XT + 2); i += blockDim.x) {
        const int c = i / (9 * (XT + 2)), rem = i % (9 * (XT + 2));
        const int dzy = rem / (XT + 2), xo = rem % (XT + 2);
        const int zz = z + dzy / 3 - 1, yy = y + dzy % 3 - 1, xx = x0 + xo - 1;
        float val = 0.f;
        if (c0 + c < ci && zz >= 0 && zz < d.nz && yy >= 0 && yy < d.ny && xx >= 0 && xx < d.nx)
          val = in[(size_t)(c0 + c) * chan + (size_t)zz * plane + (size_t)yy * d.nx + xx];
        si[c][dzy][xo] = val;
      }
      __syncthreads();
      if (active) {
        for (int x = 0; x < XT; ++x) {
          const float g = sd[o][x];
#pragma unroll
          for (int dzy = 0; dzy < 9; ++dzy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) acc[dzy * 3 + dx] = fmaf(g, si[cl][dzy][x + dx], acc[dzy * 3 + dx]);
        }
      }
    }
  }
  if (active) {
    float* p = partial + (((size_t)blockIdx.y * ci + c0 + cl) * co + o) * 27;
#pragma unroll
    for (int t = 0; t < 27; ++t) p[t] = acc[t];
  }
}

// grad_w[o][c][t] += sum_g partial[g][c][o][t]; grad_b[o] += sum_v dout[o][v]
__global__ void dw_reduce_kernel(const float* __restrict__ partial, int groups, int ci, int co,
                                 float* __restrict__ gw) {
  const size_t n = (size_t)co * ci * 27;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(i % 27);
    const int c = (int)((i / 27) % ci);
    const int o = (int)(i / (27 * (size_t)ci));
    float s = 0.f;
    for (int g = 0; g < groups; ++g) s += partial[(((size_t)g * ci + c) * co + o) * 27 + t];
    gw[i] += s;
  }
}

__global__ void db_kernel(const float* __restrict__ dout, size_t vox, float* __restrict__ gb) {
  __shared__ float red[256];
  const int o = blockIdx.x;
  float s = 0.f;
  for (size_t v = threadIdx.x; v < vox; v += blockDim.x) s += dout[(size_t)o * vox + v];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) gb[o] += red[0];
}

// ---------------------------------------------------------------------------
// pooling, upsampling, activations
// ---------------------------------------------------------------------------
__global__ void pool_kernel(const float* __restrict__ in, Dims f, float* __restrict__ out, Dims c_, int C) {
  const size_t n = (size_t)C * c_.vox();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % c_.nx), y = (int)((i / c_.nx) % c_.ny), z = (int)((i / ((size_t)c_.nx * c_.ny)) % c_.nz);
    const int ch = (int)(i / c_.vox());
    float s = 0.f;
    int cnt = 0;
    for (int oy = 0; oy < 2; ++oy)
      for (int ox = 0; ox < 2; ++ox) {
        const int yy = 2 * y + oy, xx = 2 * x + ox;
        if (yy < f.ny && xx < f.nx) {
          s += in[(size_t)ch * f.vox() + ((size_t)z * f.ny + yy) * f.nx + xx];
          ++cnt;
        }
      }
    out[i] = s / (float)cnt;
  }
}

__global__ void pool_backward_kernel(const float* __restrict__ dout, Dims c_, float* __restrict__ din, Dims f, int C,
                                     int accumulate) {
  const size_t n = (size_t)C * f.vox();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % f.nx), y = (int)((i / f.nx) % f.ny), z = (int)((i / ((size_t)f.nx * f.ny)) % f.nz);
    const int ch = (int)(i / f.vox());
    const int cy = y / 2, cx = x / 2;
    const int cnt = (2 * cy + 1 < f.ny ? 2 : 1) * (2 * cx + 1 < f.nx ? 2 : 1);
    const float g = dout[(size_t)ch * c_.vox() + ((size_t)z * c_.ny + cy) * c_.nx + cx] / (float)cnt;
    din[i] = accumulate ? din[i] + g : g;
  }
}

// out = up(coarse) + skip
__global__ void up_add_kernel(const float* __restrict__ coarse, Dims c_, const float* __restrict__ skip,
                              float* __restrict__ out, Dims f, int C) {
  const size_t n = (size_t)C * f.vox();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % f.nx), y = (int)((i / f.nx) % f.ny), z = (int)((i / ((size_t)f.nx * f.ny)) % f.nz);
    const int ch = (int)(i / f.vox());
    out[i] = coarse[(size_t)ch * c_.vox() + ((size_t)z * c_.ny + y / 2) * c_.nx + x / 2] + skip[i];
  }
}

// dcoarse = sum over the (up to 4) fine children of dfine
__global__ void up_backward_kernel(const float* __restrict__ dfine, Dims f, float* __restrict__ dcoarse, Dims c_,
                                   int C, int accumulate) {
  const size_t n = (size_t)C * c_.vox();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % c_.nx), y = (int)((i / c_.nx) % c_.ny), z = (int)((i / ((size_t)c_.nx * c_.ny)) % c_.nz);
    const int ch = (int)(i / c_.vox());
    float s = 0.f;
    for (int oy = 0; oy < 2; ++oy)
      for (int ox = 0; ox < 2; ++ox) {
        const int yy = 2 * y + oy, xx = 2 * x + ox;
        if (yy < f.ny && xx < f.nx) s += dfine[(size_t)ch * f.vox() + ((size_t)z * f.ny + yy) * f.nx + xx];
      }
    dcoarse[i] = accumulate ? dcoarse[i] + s : s;
  }
}

// g = g * (pre > 0)
__global__ void relu_backward_kernel(float* __restrict__ g, const float* __restrict__ pre, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!(pre[i] > 0.f)) g[i] = 0.f;
}

__global__ void add_kernel(float* __restrict__ a, const float* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] += b[i];
}

// ---------------------------------------------------------------------------
// input / output / loss / optimiser
// ---------------------------------------------------------------------------
template <typename V>
__global__ void sumsq_kernel(const V* __restrict__ v, size_t n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += (double)v[i].x * v[i].x + (double)v[i].y * v[i].y;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// X[c][vox]: c = 0..2 re v_c * s, 3..5 im v_c * s, 6 re chi, 7 im chi; s = sqrt(n / sum|v|^2)
template <typename V>
__global__ void pack_kernel(const V* __restrict__ v, const double2* __restrict__ chi, size_t vox,
                            const double* __restrict__ sumsq, float* __restrict__ X) {
  const double ss = *sumsq;
  const float s = ss > 0.0 ? (float)sqrt(3.0 * (double)vox / ss) : 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < vox; i += (size_t)gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const V a = v[(size_t)c * vox + i];
      X[(size_t)c * vox + i] = (float)a.x * s;
      X[(size_t)(3 + c) * vox + i] = (float)a.y * s;
    }
    X[(size_t)6 * vox + i] = (float)chi[i].x;
    X[(size_t)7 * vox + i] = (float)chi[i].y;
  }
}

// target of the network (the correction to the identity), scaled like the
// input: E[c] = re/im (e_c - r_c) * s
__global__ void pack_target_kernel(const float2* __restrict__ e, const float2* __restrict__ r, size_t vox,
                                   const double* __restrict__ sumsq_r, float* __restrict__ E) {
  const double ss = *sumsq_r;
  const float s = ss > 0.0 ? (float)sqrt(3.0 * (double)vox / ss) : 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < vox; i += (size_t)gridDim.x * blockDim.x)
    for (int c = 0; c < 3; ++c) {
      const float2 ev = e[(size_t)c * vox + i], rv = r[(size_t)c * vox + i];
      E[(size_t)c * vox + i] = (ev.x - rv.x) * s;
      E[(size_t)(3 + c) * vox + i] = (ev.y - rv.y) * s;
    }
}

// loss = sum (Y - E)^2 / sum |e s|^2 with E = (e - r) s: the error of
// z = r + Net(r) relative to e (sums accumulated in sums[0], sums[1])
__global__ void loss_sums_kernel(const float* __restrict__ Y, const float* __restrict__ E,
                                 const float2* __restrict__ e, size_t vox, const double* __restrict__ sumsq_r,
                                 double* __restrict__ sums) {
  __shared__ double r0[256], r1[256];
  const size_t n = 6 * vox;
  const double ss = *sumsq_r;
  const double s2 = ss > 0.0 ? 3.0 * (double)vox / ss : 0.0;
  double a = 0.0, b = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double d = (double)Y[i] - E[i];
    a += d * d;
  }
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * vox; i += (size_t)gridDim.x * blockDim.x)
    b += ((double)e[i].x * e[i].x + (double)e[i].y * e[i].y) * s2;
  r0[threadIdx.x] = a;
  r1[threadIdx.x] = b;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      r0[threadIdx.x] += r0[threadIdx.x + k];
      r1[threadIdx.x] += r1[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&sums[0], r0[0]);
    atomicAdd(&sums[1], r1[0]);
  }
}

// dY = 2 (Y - E) / sum E^2
__global__ void loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ E, size_t n,
                                 const double* __restrict__ sums, float* __restrict__ dY) {
  const float k = (float)(2.0 / sums[1]);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dY[i] = k * (Y[i] - E[i]);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, float scale_g) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i] * scale_g;
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    q[i] = __float2bfloat16_rn(p[i]);
}

// w'[c][o][26 - t] = w[o][c][t] for one layer (backward data)
__global__ void flip_kernel(const __nv_bfloat16* __restrict__ w, int ci, int co, __nv_bfloat16* __restrict__ wf) {
  const size_t n = (size_t)co * ci * 27;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(i % 27);
    const int c = (int)((i / 27) % ci);
    const int o = (int)(i / (27 * (size_t)ci));
    wf[((size_t)c * co + o) * 27 + (26 - t)] = w[i];
  }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static unsigned ew_blocks(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

struct NetTensors {
  Dims L[4];
  float* X;          // 8 x V0
  float* encz[4];    // 32 x V_l
  float* h[4];       // 32 x V_l
  float* a[4];       // pooled input of level l (l >= 1)
  float* decin[3];
  float* decz[3];
  float* u[3];
  float* Y;          // 6 x V0
  float* E;          // 6 x V0 (training target)
  float* dY;
  float* g1;         // 32 x V0 scratch gradients
  float* g2;
  float* dh[4];
};

static size_t tensors_floats(const Dims* L) {
  size_t t = 8 * L[0].vox() + 3 * 6 * L[0].vox() + 2 * 32 * L[0].vox();
  for (int l = 0; l < 4; ++l) t += 32 * L[l].vox() * (2 + (l >= 1) + 1);
  for (int l = 0; l < 3; ++l) t += 3 * 32 * L[l].vox();
  return t;
}

static vie_status layout(vie_net* net, const int n[3], NetTensors* T) {
  T->L[0] = Dims{n[2], n[1], n[0]};
  for (int l = 1; l < 4; ++l) T->L[l] = Dims{T->L[l - 1].nz, (T->L[l - 1].ny + 1) / 2, (T->L[l - 1].nx + 1) / 2};
  const size_t need = tensors_floats(T->L);
  if (need > net->ws_cap) {
    cudaFree(net->ws);
    net->ws = nullptr;
    net->ws_cap = 0;
    VIE_CUDA_TRY(cudaMalloc((void**)&net->ws, need * sizeof(float)));
    net->ws_cap = need;
  }
  float* p = net->ws;
  auto take = [&](size_t k) { float* r = p; p += k; return r; };
  const size_t V0 = T->L[0].vox();
  T->X = take(8 * V0);
  for (int l = 0; l < 4; ++l) {
    T->encz[l] = take(32 * T->L[l].vox());
    T->h[l] = take(32 * T->L[l].vox());
    T->a[l] = l >= 1 ? take(32 * T->L[l].vox()) : nullptr;
    T->dh[l] = take(32 * T->L[l].vox());
  }
  for (int l = 0; l < 3; ++l) {
    T->decin[l] = take(32 * T->L[l].vox());
    T->decz[l] = take(32 * T->L[l].vox());
    T->u[l] = take(32 * T->L[l].vox());
  }
  T->Y = take(6 * V0);
  T->E = take(6 * V0);
  T->dY = take(6 * V0);
  T->g1 = take(32 * V0);
  T->g2 = take(32 * V0);
  return VIE_OK;
}

// The tensor-core layouts of the BF16 weights, refreshed whenever they
// change: wpack (forward) and wpackf (the flipped transpose, for the input
// gradients of tensor-core training).
static vie_status pack_weights(vie_net* net, cudaStream_t s) {
  for (int l = 0; l < kNumLayers; ++l) {
    const int ci = kLayerDefs[l].ci, co = kLayerDefs[l].co;
    const size_t n = pack_size(l);
    pack_mma_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        net->wbf + layer_w_off(l), ci, co, tc_cpad(ci), tc_npad(co), net->wpack + pack_off(l));
    flip_kernel<<<ew_blocks((size_t)co * ci * 27), 256, 0, s>>>(net->wbf + layer_w_off(l), ci, co,
                                                                net->wflip + layer_w_off(l));
    const size_t m = packf_size(l);
    pack_mma_weights_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(net->wflip + layer_w_off(l), co, ci,
                                                                        tc_cpad(co), tc_npad(ci),
                                                                        net->wpackf + packf_off(l));
  }
  VIE_LAUNCH_CHECK();
  return VIE_OK;
}

static vie_status conv(vie_net* net, int layer, const float* in, const __nv_bfloat16* w, const float* bias, int ci,
                       int co, float* pre, float* out, Dims d, int relu, cudaStream_t s) {
  (void)net;
  (void)layer;
  const dim3 grid((unsigned)((d.nx + kConvThreads * kConvVox - 1) / (kConvThreads * kConvVox)), (unsigned)d.ny,
                  (unsigned)d.nz);
  if (co == 32)
    conv_fwd_kernel<32><<<grid, kConvThreads, 0, s>>>(in, ci, w, bias, pre, out, d, relu);
  else if (co == 6)
    conv_fwd_kernel<6><<<grid, kConvThreads, 0, s>>>(in, ci, w, bias, pre, out, d, relu);
  else if (co == 8)
    conv_fwd_kernel<8><<<grid, kConvThreads, 0, s>>>(in, ci, w, bias, pre, out, d, relu);
  else {
    set_error("unsupported channel count %d", co);
    return VIE_ERR_INVALID;
  }
  VIE_LAUNCH_CHECK();
  return VIE_OK;
}

static const __nv_bfloat16* W(vie_net* n, int l) { return n->wbf + layer_w_off(l); }
static const float* B(vie_net* n, int l) { return n->master + layer_b_off(l); }

// Training forward pass (FP32 activations); keeps every intermediate in T.
static vie_status net_forward(vie_net* net, NetTensors& T, cudaStream_t s) {
  vie_status st;
  auto cv = [&](int layer, const float* in, float* pre, float* out, Dims d, int relu) {
    return conv(net, layer, in, W(net, layer), B(net, layer), kLayerDefs[layer].ci, kLayerDefs[layer].co, pre, out,
                d, relu, s);
  };
  for (int l = 0; l < 4; ++l) {
    const float* a = T.X;
    if (l > 0) {
      pool_kernel<<<ew_blocks(32 * T.L[l].vox()), 256, 0, s>>>(T.h[l - 1], T.L[l - 1], T.a[l], T.L[l], 32);
      a = T.a[l];
    }
    st = cv(ENC0 + l, a, T.encz[l], T.h[l], T.L[l], 1);
    if (st != VIE_OK) return st;
  }
  const float* u = T.h[3];
  for (int l = 2; l >= 0; --l) {
    const int layer = DEC0 - l;   // dec2 = 4, dec1 = 5, dec0 = 6
    up_add_kernel<<<ew_blocks(32 * T.L[l].vox()), 256, 0, s>>>(u, T.L[l + 1], T.h[l], T.decin[l], T.L[l], 32);
    st = cv(layer, T.decin[l], T.decz[l], T.u[l], T.L[l], 1);
    if (st != VIE_OK) return st;
    u = T.u[l];
  }
  return cv(OUTL, T.u[0], nullptr, T.Y, T.L[0], 0);
}

// gradient of a layer's weights and bias, accumulated into net->grad
static vie_status weight_grad(vie_net* net, int layer, const float* in, const float* dout, Dims d, cudaStream_t s) {
  const int ci = kLayerDefs[layer].ci, co = kLayerDefs[layer].co;
  const int groups = 64;
  const size_t need = (size_t)groups * ci * co * 27;
  if (need > net->partial_cap) {
    cudaFree(net->partial);
    net->partial = nullptr;
    net->partial_cap = 0;
    VIE_CUDA_TRY(cudaMalloc((void**)&net->partial, need * sizeof(float)));
    net->partial_cap = need;
  }
  const int g = groups < d.nz * d.ny ? groups : d.nz * d.ny;
  conv_dw_kernel<<<dim3((unsigned)((ci + 7) / 8), (unsigned)g), 256, 0, s>>>(in, ci, dout, co, d, net->partial);
  dw_reduce_kernel<<<ew_blocks((size_t)co * ci * 27), 256, 0, s>>>(net->partial, g, ci, co,
                                                                   net->grad + layer_w_off(layer));
  db_kernel<<<co, 256, 0, s>>>(dout, d.vox(), net->grad + layer_b_off(layer));
  VIE_LAUNCH_CHECK();
  return VIE_OK;
}

// gradient of the input of a layer: conv with flipped weights (no bias)
static vie_status data_grad(vie_net* net, int layer, const float* dout, float* din, Dims d, cudaStream_t s) {
  const int ci = kLayerDefs[layer].ci, co = kLayerDefs[layer].co;
  const __nv_bfloat16* wf = net->wflip + layer_w_off(layer);
  return conv(net, layer, dout, wf, nullptr, co, ci, nullptr, din, d, 0, s);
}

// backward pass from T.dY; accumulates into net->grad
static vie_status net_backward(vie_net* net, NetTensors& T, cudaStream_t s) {
  vie_status st;
  for (int l = 0; l < kNumLayers; ++l) {
    flip_kernel<<<ew_blocks((size_t)kLayerDefs[l].co * kLayerDefs[l].ci * 27), 256, 0, s>>>(
        W(net, l), kLayerDefs[l].ci, kLayerDefs[l].co, net->wflip + layer_w_off(l));
  }
  const Dims L0 = T.L[0];
  st = weight_grad(net, OUTL, T.u[0], T.dY, L0, s);
  if (st != VIE_OK) return st;
  st = data_grad(net, OUTL, T.dY, T.g1, L0, s);      // d u0
  if (st != VIE_OK) return st;
  for (int l = 0; l < 4; ++l) cudaMemsetAsync(T.dh[l], 0, 32 * T.L[l].vox() * sizeof(float), s);
  float* du = T.g1;
  for (int l = 0; l <= 2; ++l) {
    const int layer = DEC0 - l;
    const Dims d = T.L[l];
    relu_backward_kernel<<<ew_blocks(32 * d.vox()), 256, 0, s>>>(du, T.decz[l], 32 * d.vox());
    st = weight_grad(net, layer, T.decin[l], du, d, s);
    if (st != VIE_OK) return st;
    st = data_grad(net, layer, du, T.g2, d, s);        // d decin_l
    if (st != VIE_OK) return st;
    add_kernel<<<ew_blocks(32 * d.vox()), 256, 0, s>>>(T.dh[l], T.g2, 32 * d.vox());
    // gradient to the coarse input of the upsampling: u_{l+1} (or h_3)
    float* dcoarse = (l == 2) ? T.dh[3] : T.g1;
    up_backward_kernel<<<ew_blocks(32 * T.L[l + 1].vox()), 256, 0, s>>>(T.g2, d, dcoarse, T.L[l + 1], 32,
                                                                        l == 2 ? 1 : 0);
    du = T.g1;
  }
  for (int l = 3; l >= 0; --l) {
    const Dims d = T.L[l];
    relu_backward_kernel<<<ew_blocks(32 * d.vox()), 256, 0, s>>>(T.dh[l], T.encz[l], 32 * d.vox());
    const float* a = l == 0 ? T.X : T.a[l];
    st = weight_grad(net, ENC0 + l, a, T.dh[l], d, s);
    if (st != VIE_OK) return st;
    if (l > 0) {
      st = data_grad(net, ENC0 + l, T.dh[l], T.g2, d, s);   // d a_l
      if (st != VIE_OK) return st;
      pool_backward_kernel<<<ew_blocks(32 * T.L[l - 1].vox()), 256, 0, s>>>(T.g2, d, T.dh[l - 1], T.L[l - 1], 32, 1);
    }
  }
  VIE_LAUNCH_CHECK();
  return VIE_OK;
}

// ---------------------------------------------------------------------------
// inference on the tensor cores (channels-last BF16 activations)
// ---------------------------------------------------------------------------
struct TcCache {
  int n[3] = {0, 0, 0};
  __nv_bfloat16* ws = nullptr;
  size_t cap = 0;
  Dims L[4];
  int bx[kNumLayers], by[kNumLayers];   // tile of each layer
  // h_l (l < 3, skips), pooled inputs a_l (l >= 1), decoder inputs decin_l, u_0
  __nv_bfloat16 *X = nullptr, *h[3] = {}, *a[4] = {}, *decin[3] = {}, *u0 = nullptr;
  double* norm = nullptr;       // kTcNormBlocks partial sums of |v|^2, then the total
  CUtensorMap mA[kNumLayers];   // input activation of each layer
  CUtensorMap mW[kNumLayers];   // packed weights of each layer
  bool wmaps = false;
};


static size_t tc_ws_elems(const Dims* L) {
  size_t t = 16 * L[0].vox() + 32 * L[0].vox();         // X, u_0
  for (int l = 0; l < 3; ++l) t += 2 * 32 * L[l].vox();  // h_l, decin_l
  for (int l = 1; l < 4; ++l) t += 32 * L[l].vox();      // a_l
  return t;
}

// (Re)build the workspace and the tensor maps for the grid n.
static vie_status tc_prepare(vie_net* net, const int n[3], TcCache** out) {
  if (!net->tc) net->tc = new TcCache();
  TcCache* c = net->tc;
  if (!c->norm) {   // assigned only on success, so a failed allocation is retried
    double* buf = nullptr;
    VIE_CUDA_TRY(cudaMalloc((void**)&buf, (kTcNormBlocks + 1) * sizeof(double)));
    c->norm = buf;
  }
  if (!c->wmaps) {
    for (int l = 0; l < kNumLayers; ++l) {
      vie_status st = tc_encode_w(&c->mW[l], net->wpack + pack_off(l), tc_cpad(kLayerDefs[l].ci),
                                  tc_npad(kLayerDefs[l].co));
      if (st != VIE_OK) return st;
    }
    c->wmaps = true;
  }
  if (c->ws && c->n[0] == n[0] && c->n[1] == n[1] && c->n[2] == n[2]) {
    *out = c;
    return VIE_OK;
  }
  c->L[0] = Dims{n[2], n[1], n[0]};
  for (int l = 1; l < 4; ++l) c->L[l] = Dims{c->L[l - 1].nz, (c->L[l - 1].ny + 1) / 2, (c->L[l - 1].nx + 1) / 2};
  const size_t need = tc_ws_elems(c->L);
  if (need > c->cap) {
    cudaFree(c->ws);
    c->ws = nullptr;
    c->cap = 0;
    VIE_CUDA_TRY(cudaMalloc((void**)&c->ws, need * sizeof(__nv_bfloat16)));
    c->cap = need;
  }
  __nv_bfloat16* p = c->ws;
  auto take = [&](size_t k) { __nv_bfloat16* r = p; p += k; return r; };
  c->X = take(16 * c->L[0].vox());
  c->u0 = take(32 * c->L[0].vox());
  for (int l = 0; l < 3; ++l) {
    c->h[l] = take(32 * c->L[l].vox());
    c->decin[l] = take(32 * c->L[l].vox());
  }
  c->a[0] = nullptr;
  for (int l = 1; l < 4; ++l) c->a[l] = take(32 * c->L[l].vox());
  // layer inputs: enc0 X, enc1..3 pooled a_l, dec_l decin_l, out u_0; the
  // encoders below the coarsest level pool in their epilogue (16-wide tiles)
  const __nv_bfloat16* in[kNumLayers] = {c->X, c->a[1], c->a[2], c->a[3], c->decin[2], c->decin[1], c->decin[0], c->u0};
  for (int l = 0; l < kNumLayers; ++l) {
    tc_pick_tile(c->L[kLayerLevel[l]], l <= ENC2, &c->bx[l], &c->by[l]);
    vie_status st = tc_encode_act(&c->mA[l], in[l], l == ENC0 ? 16 : 32, c->L[kLayerLevel[l]], c->bx[l], c->by[l]);
    if (st != VIE_OK) return st;
  }
  c->n[0] = n[0];
  c->n[1] = n[1];
  c->n[2] = n[2];
  *out = c;
  return VIE_OK;
}

static void tc_free(TcCache* c) {
  if (!c) return;
  cudaFree(c->ws);
  cudaFree(c->norm);
  delete c;
}

// Inference: |v|^2 and the packed input, then eight convolutions whose
// epilogues also pool (enc0..enc2) or upsample and add the skip (enc3, dec2,
// dec1); the output layer's epilogue forms z = v + Net(v) / s.
template <typename V>
static vie_status net_apply_t(vie_net* net, const vie_plan* p, const V* v, V* z, cudaStream_t s) {
  TcCache* c = nullptr;
  vie_status st = tc_prepare(net, p->n, &c);
  if (st != VIE_OK) return st;
  double* sumsq = c->norm + kTcNormBlocks;
  st = tc_pack_input<V>(v, p->chi64, c->L[0], c->norm, c->X, s);
  if (st != VIE_OK) return st;
  auto conv = [&](int layer, int mode, __nv_bfloat16* out, __nv_bfloat16* out2, int level2,
                  const __nv_bfloat16* skip) {
    TcConvArgs a{};
    a.d = c->L[kLayerLevel[layer]];
    a.d2 = level2 >= 0 ? c->L[level2] : a.d;
    a.bx = c->bx[layer];
    a.by = c->by[layer];
    a.bias = B(net, layer);
    a.co = kLayerDefs[layer].co;
    a.out = out;
    a.out2 = out2;
    a.skip = skip;
    a.v = v;
    a.z = z;
    a.sumsq = sumsq;
    a.bad = net->bad;
    return tc_conv(c->mA[layer], c->mW[layer], tc_cpad(kLayerDefs[layer].ci), tc_npad(kLayerDefs[layer].co), mode,
                   a, s);
  };
  for (int l = 0; l < 3; ++l)
    if ((st = conv(ENC0 + l, TC_RELU_POOL, c->h[l], c->a[l + 1], l + 1, nullptr)) != VIE_OK) return st;
  if ((st = conv(ENC3, TC_RELU_UPADD, nullptr, c->decin[2], 2, c->h[2])) != VIE_OK) return st;
  if ((st = conv(DEC2, TC_RELU_UPADD, nullptr, c->decin[1], 1, c->h[1])) != VIE_OK) return st;
  if ((st = conv(DEC1, TC_RELU_UPADD, nullptr, c->decin[0], 0, c->h[0])) != VIE_OK) return st;
  if ((st = conv(DEC0, TC_RELU_BF16, c->u0, nullptr, -1, nullptr)) != VIE_OK) return st;
  return conv(OUTL, sizeof(V) == 8 ? TC_UNPACK_C64 : TC_UNPACK_C128, nullptr, nullptr, -1, nullptr);
}

// The preconditioner set on a plan: a network (learned) or a block-circulant
// matrix (Sec. 5.4); exactly one of net and circ is set.
struct PrecondCtx {
  vie_net* net;
  const vie_plan* plan;
  vie_circulant* circ;
  bool owns_net;              // the network was built by vie_set_preconditioner from caller weights
};

static vie_status precond_apply(void* ctx, int dtype, const void* v, void* z, cudaStream_t s) {
  PrecondCtx* c = (PrecondCtx*)ctx;
  if (c->circ) return circulant_apply(c->circ, dtype, v, z, s);
  if (dtype == VIE_C64) return net_apply_t<float2>(c->net, c->plan, (const float2*)v, (float2*)z, s);
  return net_apply_t<double2>(c->net, c->plan, (const double2*)v, (double2*)z, s);
}

void free_precond(vie_plan* p) {
  if (p && p->precond) {
    PrecondCtx* c = (PrecondCtx*)p->precond;
    if (c->owns_net) vie_net_destroy(c->net);
    delete c;
    p->precond = nullptr;
  }
}

vie_status precond_get(vie_plan* p, vie_precond_fn* fn, void** ctx) {
  if (!p->precond) {
    *fn = nullptr;
    *ctx = nullptr;
    set_error("no preconditioner has been set on this plan");
    return VIE_ERR_INVALID;
  }
  *fn = precond_apply;
  *ctx = p->precond;
  return VIE_OK;
}

int precond_is_learned(const vie_plan* p) {
  return (p && p->precond && ((PrecondCtx*)p->precond)->net) ? 1 : 0;
}

int precond_fallback_flag(vie_plan* p, int clear) {
  if (!p || !p->precond) return 0;
  PrecondCtx* c = (PrecondCtx*)p->precond;
  if (!c->net) return 0;
  int h = 0;
  cudaMemcpy(&h, c->net->bad, sizeof(int), cudaMemcpyDeviceToHost);
  if (clear && h) cudaMemset(c->net->bad, 0, sizeof(int));
  return h;
}

}  // namespace vie

using namespace vie;

extern "C" {

vie_status vie_net_create(vie_net** out, const float* params_host, size_t count, unsigned long long seed) {
  clear_error();
  if (!out) { set_error("null argument"); return VIE_ERR_INVALID; }
  *out = nullptr;
  const size_t np = total_params();
  if (params_host && count != np) {
    set_error("expected %zu parameters, got %zu", np, count);
    return VIE_ERR_INVALID;
  }
  vie_net* n = new vie_net();
  VIE_CUDA_TRY(cudaGetDevice(&n->device));
  n->nparams = np;
  std::vector<float> h(np);
  if (params_host) {
    memcpy(h.data(), params_host, np * sizeof(float));
  } else {
    // He initialisation from a 64-bit linear congruential generator (Box-Muller)
    unsigned long long st = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto uni = [&]() {
      st = st * 6364136223846793005ULL + 1442695040888963407ULL;
      return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < kNumLayers; ++l) {
      const double sd = sqrt(2.0 / (27.0 * kLayerDefs[l].ci));
      const size_t nw = (size_t)kLayerDefs[l].co * kLayerDefs[l].ci * 27;
      for (size_t i = 0; i < nw; ++i) {
        const double u1 = uni(), u2 = uni();
        h[layer_w_off(l) + i] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2));
      }
      for (int o = 0; o < kLayerDefs[l].co; ++o) h[layer_b_off(l) + o] = 0.f;
    }
    // output layer at zero: the untrained preconditioner is the identity
    for (size_t i = 0; i < (size_t)kLayerDefs[OUTL].co * kLayerDefs[OUTL].ci * 27; ++i) h[layer_w_off(OUTL) + i] = 0.f;
  }
  struct { void** p; size_t sz; } a[] = {
      {(void**)&n->master, np * 4}, {(void**)&n->grad, np * 4}, {(void**)&n->m1, np * 4}, {(void**)&n->m2, np * 4},
      {(void**)&n->wbf, np * 2},    {(void**)&n->wflip, np * 2}, {(void**)&n->scal, 8 * sizeof(double)},
      {(void**)&n->wpack, pack_off(kNumLayers) * 2}, {(void**)&n->wpackf, packf_off(kNumLayers) * 2},
      {(void**)&n->bad, sizeof(int)}};
  for (auto& e : a) {
    cudaError_t err = cudaMalloc(e.p, e.sz);
    if (err != cudaSuccess) {
      set_error("network cudaMalloc: %s", cudaGetErrorString(err));
      vie_net_destroy(n);
      return VIE_ERR_OOM;
    }
  }
  cudaMemcpy(n->master, h.data(), np * 4, cudaMemcpyHostToDevice);
  cudaMemset(n->grad, 0, np * 4);
  cudaMemset(n->m1, 0, np * 4);
  cudaMemset(n->m2, 0, np * 4);
  cudaMemset(n->bad, 0, sizeof(int));
  to_bf16_kernel<<<ew_blocks(np), 256>>>(n->master, n->wbf, np);
  pack_weights(n, 0);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_error("network init: %s", cudaGetErrorString(e));
    vie_net_destroy(n);
    return VIE_ERR_CUDA;
  }
  *out = n;
  return VIE_OK;
}

vie_status vie_net_destroy(vie_net* n) {
  if (!n) return VIE_OK;
  cudaFree(n->master); cudaFree(n->grad); cudaFree(n->m1); cudaFree(n->m2); cudaFree(n->wbf); cudaFree(n->wflip);
  cudaFree(n->wpack); cudaFree(n->wpackf);
  cudaFree(n->ws); cudaFree(n->partial); cudaFree(n->scal); cudaFree(n->bad);
  tc_free(n->tc);
  tc_train_free(n->train);
  delete n;
  return VIE_OK;
}

size_t vie_net_param_count(void) { return total_params(); }

vie_status vie_net_get_params(const vie_net* n, float* out_host) {
  clear_error();
  if (!n || !out_host) { set_error("null argument"); return VIE_ERR_INVALID; }
  VIE_CUDA_TRY(cudaMemcpy(out_host, n->master, n->nparams * 4, cudaMemcpyDeviceToHost));
  return VIE_OK;
}

vie_status vie_net_get_grads(const vie_net* n, float* out_host) {
  clear_error();
  if (!n || !out_host) { set_error("null argument"); return VIE_ERR_INVALID; }
  VIE_CUDA_TRY(cudaMemcpy(out_host, n->grad, n->nparams * 4, cudaMemcpyDeviceToHost));
  return VIE_OK;
}

vie_status vie_net_apply(vie_net* n, const vie_plan* p, const void* v_dev, void* z_dev, int dtype, void* stream) {
  clear_error();
  if (!n || !p || !v_dev || !z_dev) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (dtype != VIE_C64 && dtype != VIE_C128) { set_error("dtype must be VIE_C64 or VIE_C128"); return VIE_ERR_INVALID; }
  PrecondCtx c{n, p, nullptr, false};
  return precond_apply(&c, dtype, v_dev, z_dev, (cudaStream_t)stream);
}

vie_status vie_net_accumulate(vie_net* n, const vie_plan* p, const void* r_dev, const void* e_dev, double* loss,
                              void* stream) {
  clear_error();
  if (!n || !p || !r_dev || !e_dev) { set_error("null argument"); return VIE_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  if (n->train_mode == VIE_TRAIN_TENSOR_BF16) {
    TcTrainParams P{n->wpack, n->wpackf, n->master, n->grad, n->bad};
    double l = 0.0;
    vie_status st = tc_train_accumulate(&n->train, P, p->n, p->chi64, (const float2*)r_dev, (const float2*)e_dev, &l, s);
    if (loss) *loss = l;
    return st;
  }
  NetTensors T;
  vie_status st = layout(n, p->n, &T);
  if (st != VIE_OK) return st;
  const size_t V0 = T.L[0].vox();
  double* scal = (double*)n->scal;
  VIE_CUDA_TRY(cudaMemsetAsync(scal, 0, 4 * sizeof(double), s));
  sumsq_kernel<float2><<<ew_blocks(3 * V0), 256, 0, s>>>((const float2*)r_dev, 3 * V0, scal);
  pack_kernel<float2><<<ew_blocks(V0), 256, 0, s>>>((const float2*)r_dev, p->chi64, V0, scal, T.X);
  pack_target_kernel<<<ew_blocks(V0), 256, 0, s>>>((const float2*)e_dev, (const float2*)r_dev, V0, scal, T.E);
  VIE_LAUNCH_CHECK();
  st = net_forward(n, T, s);
  if (st != VIE_OK) return st;
  loss_sums_kernel<<<ew_blocks(6 * V0), 256, 0, s>>>(T.Y, T.E, (const float2*)e_dev, V0, scal, scal + 1);
  loss_grad_kernel<<<ew_blocks(6 * V0), 256, 0, s>>>(T.Y, T.E, 6 * V0, scal + 1, T.dY);
  VIE_LAUNCH_CHECK();
  st = net_backward(n, T, s);
  if (st != VIE_OK) return st;
  double h[3] = {0, 0, 0};
  VIE_CUDA_TRY(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (loss) *loss = h[2] > 0 ? h[1] / h[2] : 0.0;
  return VIE_OK;
}

vie_status vie_net_set_training(vie_net* n, int mode) {
  clear_error();
  if (!n) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (mode != VIE_TRAIN_TENSOR_BF16 && mode != VIE_TRAIN_FP32) {
    set_error("training mode must be VIE_TRAIN_TENSOR_BF16 or VIE_TRAIN_FP32");
    return VIE_ERR_INVALID;
  }
  n->train_mode = mode;
  return VIE_OK;
}

vie_status vie_net_zero_grad(vie_net* n) {
  clear_error();
  if (!n) { set_error("null argument"); return VIE_ERR_INVALID; }
  VIE_CUDA_TRY(cudaMemset(n->grad, 0, n->nparams * 4));
  return VIE_OK;
}

vie_status vie_net_adam_step(vie_net* n, float lr, float grad_scale, void* stream) {
  clear_error();
  if (!n) { set_error("null argument"); return VIE_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
  adam_kernel<<<ew_blocks(n->nparams), 256, 0, s>>>(n->master, n->grad, n->m1, n->m2, n->nparams, lr, b1, b2, 1e-8f,
                                                    c1, c2, grad_scale);
  to_bf16_kernel<<<ew_blocks(n->nparams), 256, 0, s>>>(n->master, n->wbf, n->nparams);
  VIE_LAUNCH_CHECK();
  vie_status st = pack_weights(n, s);
  if (st != VIE_OK) return st;
  VIE_CUDA_TRY(cudaMemsetAsync(n->grad, 0, n->nparams * 4, s));
  return VIE_OK;
}

vie_status vie_net_status(vie_net* n, int* flag, int clear) {
  clear_error();
  if (!n || !flag) { set_error("null argument"); return VIE_ERR_INVALID; }
  VIE_CUDA_TRY(cudaMemcpy(flag, n->bad, sizeof(int), cudaMemcpyDeviceToHost));
  if (clear) VIE_CUDA_TRY(cudaMemset(n->bad, 0, sizeof(int)));
  return VIE_OK;
}

vie_status vie_set_preconditioner_net(vie_plan* p, vie_net* n) {
  clear_error();
  if (!p) { set_error("null plan"); return VIE_ERR_INVALID; }
  free_precond(p);
  if (n) p->precond = new PrecondCtx{n, p, nullptr, false};
  return VIE_OK;
}

vie_status vie_set_preconditioner(vie_plan* p, const void* weights, size_t bytes) {
  clear_error();
  if (!p) { set_error("null plan"); return VIE_ERR_INVALID; }
  if (!weights) {
    free_precond(p);
    return VIE_OK;
  }
  const size_t np = total_params();
  if (bytes != np * sizeof(float)) {
    set_error("weights must hold %zu bytes (%zu FP32 parameters), got %zu", np * sizeof(float), np, bytes);
    return VIE_ERR_INVALID;
  }
  int cur = -1;
  VIE_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != p->device) { set_error("the plan's device (%d) must be current", p->device); return VIE_ERR_INVALID; }
  vie_net* n = nullptr;
  vie_status st = vie_net_create(&n, (const float*)weights, np, 0);
  if (st != VIE_OK) return st;
  free_precond(p);
  p->precond = new PrecondCtx{n, p, nullptr, true};
  return VIE_OK;
}

vie_status vie_set_circulant_preconditioner(vie_plan* p, vie_circulant* c) {
  clear_error();
  if (!p) { set_error("null plan"); return VIE_ERR_INVALID; }
  if (c && circulant_plan(c) != p) {
    // the factors depend on the grid and contrast of the plan they were built for
    set_error("the block-circulant preconditioner belongs to another plan");
    return VIE_ERR_INVALID;
  }
  free_precond(p);
  if (c) p->precond = new PrecondCtx{nullptr, p, c, false};
  return VIE_OK;
}

}  // extern "C"
