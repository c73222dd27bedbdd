// Tensor-core training path of the learned preconditioner: BF16 weights
// and channels-last BF16 activations, FP32 accumulation in tensor memory.
//
// Forward: the inference convolutions (conv_tc.cu) with epilogues that keep
// every tensor the backward pass needs (the coarse ReLU outputs of enc3,
// dec2 and dec1 besides their upsampled sums, and the network output in
// FP32).
//
// Backward, per layer from the output down:
//   input gradient   the same tensor-core convolution with the flipped,
//                    transposed weights (TC_GRAD_BF16), masked by the ReLU
//                    of the layer's input where that input is a ReLU output;
//   weight gradient  dW[t][o][c] = sum_p dPre[p][o] In[p + t - 1][c], a GEMM
//                    over the positions p (dw_tc_kernel below);
//   bias gradient    db[o] = sum_p dPre[p][o] (summed while the GEMM operands
//                    are written);
// and element-wise steps for the upsampling (sum of the 2 x 2 children) and
// the pooling (a quarter, half or all of the parent's gradient), each with
// the ReLU mask of the tensor it produces the gradient of.
//
// The weight-gradient GEMM: for a chunk of 64 positions along x of one
// (z, y) row, A is 128 x 64 (rows dx * 32 + o: the output gradient shifted
// by dx - 1 along x, written planar by dw_operands_kernel) and, for each
// of the nine (dz, dy) taps, B is C x 64 (the layer input of row
// (z + dz - 1, y + dy - 1), planar, the TMA zero-filling rows outside the
// grid).  Nine accumulators of 128 x C in tensor memory collect a CTA's
// chunks; the epilogue writes them as per-CTA partial sums, reduced by
// dw_reduce_kernel into the FP32 gradient.
#include <cuda_bf16.h>
#include <stdio.h>

#include "net.cuh"
#include "tc.cuh"

namespace vie {

constexpr int kDwChunk = 64;       // positions along x per K chunk
constexpr int kDwMaxStages = 8;
constexpr int kDwThreads = 192;
constexpr int kDwMinChunks = 4;    // chunks per CTA at least, where the level allows

// ---------------------------------------------------------------------------
// planar operands of the weight-gradient GEMM
// ---------------------------------------------------------------------------
// The two operands in one launch (grid.x = 2 x the chunks per row; blocks
// below nxc write A, the others B), one block per (64-position chunk, y, z);
// rows are `plane` elements apart (the level-0 plane at every level):
//   A[dx * 32 + o][z][y][x] = g[z][y][x - dx + 1][o] for dx < 3, o < NPo and
//     0 <= x - dx + 1 < nx, x < nx; 0 elsewhere (rows 96..127 are zeroed
//     once when the buffer is laid out and never written);
//   B[c][z][y][x] = in[z][y][x][c] for x < nx, 0 for nx <= x < nxp;
// and the A blocks add their chunk's sum of g over positions to the bias
// gradient gb[o] (o < co).
__global__ void __launch_bounds__(256) dw_operands_kernel(const __nv_bfloat16* __restrict__ g, int NPo, int co,
                                                          const __nv_bfloat16* __restrict__ in, int C, Dims d,
                                                          int nxp, int nxc, size_t plane, __nv_bfloat16* __restrict__ A,
                                                          __nv_bfloat16* __restrict__ B, float* __restrict__ gb) {
  __shared__ __nv_bfloat16 t[kDwChunk + 2][33];
  __shared__ float bsum[8][33];
  const bool isA = (int)blockIdx.x < nxc;
  const int x0 = (isA ? blockIdx.x : blockIdx.x - nxc) * kDwChunk, y = blockIdx.y, z = blockIdx.z;
  const size_t row = (size_t)z * d.ny + y;
  const size_t base = row * nxp + x0;
  if (isA) {
    float acc = 0.f;   // thread (j, o) sums g over its positions j = tid >> 5, + 8, ...
    for (int i = threadIdx.x; i < (kDwChunk + 2) * 32; i += blockDim.x) {
      const int j = i >> 5, o = i & 31;
      const int x = x0 - 1 + j;
      __nv_bfloat16 v = __float2bfloat16_rn(0.f);
      if (o < NPo && x >= 0 && x < d.nx) v = g[(row * d.nx + x) * NPo + o];
      t[j][o] = v;
      if (j >= 1 && j <= kDwChunk) acc += __bfloat162float(v);   // positions x0 .. x0 + 63 of this chunk
    }
    bsum[threadIdx.x >> 5][threadIdx.x & 31] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      float sum = 0.f;
      for (int k = 0; k < 8; ++k) sum += bsum[k][threadIdx.x];
      if (threadIdx.x < co) atomicAdd(gb + threadIdx.x, sum);
    }
    for (int i = threadIdx.x; i < 96 * kDwChunk; i += blockDim.x) {
      const int r = i / kDwChunk, xl = i - r * kDwChunk;
      const int dx = r >> 5, o = r & 31;
      __nv_bfloat16 v = __float2bfloat16_rn(0.f);
      if (x0 + xl < d.nx) v = t[xl - dx + 2][o];
      A[r * plane + base + xl] = v;
    }
  } else {
    for (int i = threadIdx.x; i < kDwChunk * C; i += blockDim.x) {
      const int j = i / C, c = i - j * C;
      const int x = x0 + j;
      t[j][c] = x < d.nx ? in[(row * d.nx + x) * C + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C * kDwChunk; i += blockDim.x) {
      const int c = i / kDwChunk, xl = i - c * kDwChunk;
      B[c * plane + base + xl] = t[xl][c];
    }
  }
}

// ---------------------------------------------------------------------------
// weight-gradient GEMM on the tensor cores
// ---------------------------------------------------------------------------
struct DwArgs {
  Dims d;
  int nxc;            // chunks per (z, y) row
  int stages;
  float* partial;     // [gridDim.x][27][32][C]
  int* bad;
};

template <int C>
__global__ void __launch_bounds__(kDwThreads, 1) dw_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB,
                                                              const DwArgs a) {
  constexpr uint32_t ABYTES = 128 * 128;          // 128 rows x 64 positions (BF16)
  constexpr uint32_t BBYTES = C * 128;            // C rows x 64 positions
  constexpr uint32_t SBYTES = ABYTES + 9 * BBYTES;
  constexpr uint32_t NCOLS = 9 * C <= 256 ? 256 : 512;
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, C);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t S = (uint32_t)a.stages;
  uint64_t* full = (uint64_t*)(base + S * SBYTES);
  uint64_t* empty = full + kDwMaxStages;
  uint64_t* done = empty + kDwMaxStages;
  uint32_t* tslot = (uint32_t*)(done + 1);
  volatile int* abort = (volatile int*)(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long nchunks = (long)a.d.nz * a.d.ny * a.nxc;
  // balanced contiguous ranges: every CTA has at least one chunk (grid <= nchunks)
  const long k0 = (long)blockIdx.x * nchunks / gridDim.x;
  const long k1 = (long)(blockIdx.x + 1) * nchunks / gridDim.x;

  if (threadIdx.x == 0) {
    for (uint32_t i = 0; i < S; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tslot, NCOLS);
    tc::fence_before_sync();
  }
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    tc::prefetch_tensormap(&tmA);
    tc::prefetch_tensormap(&tmB);
    uint32_t it = 0;
    for (long k = k0; k < k1 && !*abort; ++k, ++it) {
      const int xc = (int)(k % a.nxc);
      const long row = k / a.nxc;
      const int y = (int)(row % a.d.ny), z = (int)(row / a.d.ny);
      const uint32_t stage = it % S, round = it / S;
      if (!tc::mbar_wait(&empty[stage], (round & 1) ^ 1, abort)) break;
      tc::mbar_arrive_expect_tx(&full[stage], SBYTES);
      unsigned char* st = base + stage * SBYTES;
      tc::tma_load_4d(st, &tmA, &full[stage], xc * kDwChunk, y, z, 0);
      for (int t = 0; t < 9; ++t)
        tc::tma_load_4d(st + ABYTES + t * BBYTES, &tmB, &full[stage], xc * kDwChunk, y + t % 3 - 1, z + t / 3 - 1, 0);
    }
    if (*abort) {
      // let the copies already issued land before the CTA exits
      for (uint32_t j = 0; j < S && j < it; ++j) {
        const uint32_t last = it - 1 - j;
        volatile int never = 0;
        tc::mbar_wait(&full[last % S], (last / S) & 1, &never);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    uint32_t it = 0;
    for (long k = k0; k < k1 && !*abort; ++k, ++it) {
      const uint32_t stage = it % S, round = it / S;
      if (!tc::mbar_wait(&full[stage], round & 1, abort)) break;
      tc::fence_after_sync();
      unsigned char* st = base + stage * SBYTES;
      const uint64_t dA = tc::smem_desc(tc::smem_u32(st), 128);
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const uint64_t dB = tc::smem_desc(tc::smem_u32(st + ABYTES + t * BBYTES), 128);
#pragma unroll
        for (int kk = 0; kk < kDwChunk / 16; ++kk)
          tc::mma_bf16(tmem + (uint32_t)(t * C), tc::desc_add(dA, 32 * kk), tc::desc_add(dB, 32 * kk), IDESC,
                       (k != k0 || kk != 0) ? 1u : 0u);
      }
      tc::mma_commit(&empty[stage]);   // frees the stage when these MMAs are done
    }
    tc::mma_commit(done);              // every MMA issued above has completed
    if (*abort) {
      // the epilogue gave up: let the MMAs in flight finish before the
      // tensor memory is released
      volatile int never = 0;
      tc::mbar_wait(done, 0, &never);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;            // tensor-memory lanes 32 q .. 32 q + 31: rows dx = q, o = lane
    const bool ok = tc::mbar_wait(done, 0, abort);
    if (__all_sync(0xffffffffu, ok) && q < 3) {
      tc::fence_after_sync();
      const uint32_t lane_base = (uint32_t)(32 * q) << 16;
#pragma unroll 1
      for (int t = 0; t < 9; ++t) {
        float v[C];
        if constexpr (C == 32) tc::tmem_ld32(tmem + lane_base + (uint32_t)(t * C), v);
        else tc::tmem_ld16(tmem + lane_base + (uint32_t)(t * C), v);
        float4* dst = reinterpret_cast<float4*>(a.partial + (((size_t)blockIdx.x * 27 + 3 * t + q) * 32 + lane) * C);
#pragma unroll
        for (int i = 0; i < C / 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort) atomicExch(a.bad, 2);
  if (warp == 1) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, NCOLS);
  }
}

// grad[(o ci + c) 27 + t] += sum_b partial[b][t][o][c]: thread i runs over
// the partial layout (t, o, c) so that the reads of every b are coalesced,
// blockIdx.y takes every gridDim.y-th b and adds its share atomically
__global__ void dw_reduce_kernel(const float* __restrict__ partial, int nb, int C, int ci, int co,
                                 float* __restrict__ grad) {
  const int n = 27 * 32 * C;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = i % C, o = (i / C) % 32, t = i / (32 * C);
  if (o >= co || c >= ci) return;
  float acc = 0.f;
#pragma unroll 4
  for (int b = blockIdx.y; b < nb; b += gridDim.y) acc += partial[(size_t)b * n + i];
  atomicAdd(grad + (o * ci + c) * 27 + t, acc);
}

// ---------------------------------------------------------------------------
// element-wise backward steps (channels-last, 32 channels, 8 per thread)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ld8(const __nv_bfloat16* p, float (&f)[8]) {
  const uint4 w = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 v = __bfloat1622float2(h[k]);
    f[2 * k] = v.x;
    f[2 * k + 1] = v.y;
  }
}
__device__ __forceinline__ void st8(__nv_bfloat16* p, const float (&f)[8]) {
  uint4 w;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
  *reinterpret_cast<uint4*>(p) = w;
}

// out[p] = (mask[p] > 0) * sum over the fine children f of p of dfine[f]
// (the gradient through out2[f] = up(u)[f] + skip[f] to the coarse ReLU
// output u = mask, then through the ReLU)
__global__ void upback_mask_kernel(const __nv_bfloat16* __restrict__ dfine, Dims f,
                                   const __nv_bfloat16* __restrict__ mask, Dims c, __nv_bfloat16* __restrict__ out) {
  const size_t n = c.vox() * 4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i >> 2;
    const int g = (int)(i & 3) * 8;
    const int x = (int)(v % c.nx), y = (int)((v / c.nx) % c.ny), z = (int)(v / ((size_t)c.nx * c.ny));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int oy = 0; oy < 2; ++oy) {
      const int fy = 2 * y + oy;
      if (fy >= f.ny) continue;
      for (int ox = 0; ox < 2; ++ox) {
        const int fx = 2 * x + ox;
        if (fx >= f.nx) continue;
        float t[8];
        ld8(dfine + (((size_t)z * f.ny + fy) * f.nx + fx) * 32 + g, t);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += t[k];
      }
    }
    float m[8];
    ld8(mask + v * 32 + g, m);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = m[k] > 0.f ? acc[k] : 0.f;
    st8(out + v * 32 + g, acc);
  }
}

// out[f] = (mask[f] > 0) * (dskip[f] + dcoarse[parent(f)] / count(parent(f)))
// (the skip and the pooled copy of the fine ReLU output mask: the pooling
// averages the 1, 2 or 4 children that exist)
__global__ void poolback_mask_kernel(const __nv_bfloat16* __restrict__ dskip, const __nv_bfloat16* __restrict__ dcoarse,
                                     Dims c, const __nv_bfloat16* __restrict__ mask, Dims f,
                                     __nv_bfloat16* __restrict__ out) {
  const size_t n = f.vox() * 4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i >> 2;
    const int g = (int)(i & 3) * 8;
    const int x = (int)(v % f.nx), y = (int)((v / f.nx) % f.ny), z = (int)(v / ((size_t)f.nx * f.ny));
    const int px = x >> 1, py = y >> 1;
    const int cx = (2 * px + 1 < f.nx) ? 2 : 1, cy = (2 * py + 1 < f.ny) ? 2 : 1;
    const float r = 1.f / (float)(cx * cy);
    float a[8], b[8], m[8];
    ld8(dskip + v * 32 + g, a);
    ld8(dcoarse + (((size_t)z * c.ny + py) * c.nx + px) * 32 + g, b);
    ld8(mask + v * 32 + g, m);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = m[k] > 0.f ? a[k] + b[k] * r : 0.f;
    st8(out + v * 32 + g, a);
  }
}

// ---------------------------------------------------------------------------
// loss on the channels-last FP32 output
// ---------------------------------------------------------------------------
// sums[0] += sum (Y - E)^2, sums[1] += sum |e s|^2 with E = (e - r) s over
// the six real channels (re x, y, z then im x, y, z); s = sqrt(3 V / ss).
__global__ void __launch_bounds__(256) loss_cl_kernel(const float* __restrict__ Y, const float2* __restrict__ e,
                                                      const float2* __restrict__ r, size_t vox,
                                                      const double* __restrict__ ss_r, double* __restrict__ sums) {
  __shared__ double r0[256], r1[256];
  const double ss = *ss_r;
  const float s = ss > 0.0 ? (float)sqrt(3.0 * (double)vox / ss) : 0.f;
  double a = 0.0, b = 0.0;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < vox; v += (size_t)gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const float2 ev = e[(size_t)c * vox + v], rv = r[(size_t)c * vox + v];
      const double dre = (double)Y[v * 16 + c] - (double)((ev.x - rv.x) * s);
      const double dim = (double)Y[v * 16 + 3 + c] - (double)((ev.y - rv.y) * s);
      a += dre * dre + dim * dim;
      b += ((double)ev.x * ev.x + (double)ev.y * ev.y) * (double)s * s;
    }
  }
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

// dY[v][k] = 2 (Y - E) / sums[1] for the six real channels, 0 for 6..15
__global__ void loss_grad_cl_kernel(const float* __restrict__ Y, const float2* __restrict__ e,
                                    const float2* __restrict__ r, size_t vox, const double* __restrict__ ss_r,
                                    const double* __restrict__ sums, __nv_bfloat16* __restrict__ dY) {
  const double ss = *ss_r;
  const float s = ss > 0.0 ? (float)sqrt(3.0 * (double)vox / ss) : 0.f;
  const float kk = sums[1] > 0.0 ? (float)(2.0 / sums[1]) : 0.f;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < vox; v += (size_t)gridDim.x * blockDim.x) {
    float d[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) d[k] = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 ev = e[(size_t)c * vox + v], rv = r[(size_t)c * vox + v];
      d[c] = kk * (Y[v * 16 + c] - (ev.x - rv.x) * s);
      d[3 + c] = kk * (Y[v * 16 + 3 + c] - (ev.y - rv.y) * s);
    }
    float lo[8], hi[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      lo[k] = d[k];
      hi[k] = d[8 + k];
    }
    st8(dY + v * 16, lo);
    st8(dY + v * 16 + 8, hi);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct TcTrain {
  int n[3] = {0, 0, 0};
  Dims L[4];
  __nv_bfloat16* ws = nullptr;
  size_t cap = 0;
  // forward: X, enc outputs h_l, pooled inputs a_l (l >= 1), decoder inputs
  // decin_l, coarse decoder outputs u_l (u_0 the output layer's input)
  __nv_bfloat16 *X = nullptr, *h[4] = {}, *a[4] = {}, *decin[3] = {}, *u[3] = {};
  // backward: dY (16 channels), per layer the gradient of its pre-activation
  // dpre[l], the input gradients of the decoders (ddecin_l) and encoders (da_l)
  __nv_bfloat16 *dY = nullptr, *dpre[kNumLayers] = {}, *ddecin[3] = {}, *da[4] = {};
  __nv_bfloat16 *Apl = nullptr, *Bpl = nullptr;   // planar GEMM operands (level 0 size)
  size_t plane0 = 0;                               // their row stride (elements)
  float* Yf = nullptr;                             // network output [V0][16]
  size_t yf_cap = 0;
  float* partial = nullptr;                        // [sms][27][32][32]
  double* norm = nullptr;                          // kTcNormBlocks + 1 partial sums of |r|^2, then loss sums
  int bxf[kNumLayers], byf[kNumLayers];            // forward tiles
  int bxb[kNumLayers], byb[kNumLayers];            // backward-data tiles
  CUtensorMap mA[kNumLayers], mW[kNumLayers];      // forward input / weights
  CUtensorMap mG[kNumLayers], mWf[kNumLayers];     // backward-data input (the layer's output gradient) / weights
  CUtensorMap mPa[kNumLayers], mPb[kNumLayers];    // weight-gradient operands
  int sms = 0, smem_optin = 0;
  const void* wpack_enc = nullptr;                 // weights the maps mW / mWf point at
  const void* wpackf_enc = nullptr;
};

static int nxp_of(int nx) { return (nx + kDwChunk - 1) / kDwChunk * kDwChunk; }

void tc_train_free(TcTrain* t) {
  if (!t) return;
  cudaFree(t->ws);
  cudaFree(t->Yf);
  cudaFree(t->partial);
  cudaFree(t->norm);
  delete t;
}

static vie_status tc_train_prepare(TcTrain** pt, const TcTrainParams& P, const int n[3]) {
  if (!*pt) *pt = new TcTrain();
  TcTrain* T = *pt;
  // keyed on the buffers, so that a failed allocation is retried next time
  if (!T->partial || !T->norm) {
    int dev = 0;
    VIE_CUDA_TRY(cudaGetDevice(&dev));
    VIE_CUDA_TRY(cudaDeviceGetAttribute(&T->sms, cudaDevAttrMultiProcessorCount, dev));
    VIE_CUDA_TRY(cudaDeviceGetAttribute(&T->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (!T->partial) {
      float* buf = nullptr;
      VIE_CUDA_TRY(cudaMalloc((void**)&buf, (size_t)T->sms * 27 * 32 * 32 * sizeof(float)));
      T->partial = buf;
    }
    if (!T->norm) {
      double* buf = nullptr;
      VIE_CUDA_TRY(cudaMalloc((void**)&buf, (kTcNormBlocks + 4) * sizeof(double)));
      T->norm = buf;
    }
  }
  const bool same = T->ws && T->n[0] == n[0] && T->n[1] == n[1] && T->n[2] == n[2];
  if (!same) {
    T->L[0] = Dims{n[2], n[1], n[0]};
    for (int l = 1; l < 4; ++l) T->L[l] = Dims{T->L[l - 1].nz, (T->L[l - 1].ny + 1) / 2, (T->L[l - 1].nx + 1) / 2};
    const size_t V0 = T->L[0].vox();
    size_t need = 16 * V0 + 16 * V0;                              // X, dY
    for (int l = 0; l < 4; ++l) need += 32 * T->L[l].vox() * 2;   // h_l, da_l
    for (int l = 1; l < 4; ++l) need += 32 * T->L[l].vox();       // a_l
    for (int l = 0; l < 3; ++l) need += 32 * T->L[l].vox() * 3;   // decin_l, u_l, ddecin_l
    for (int l = 0; l < kNumLayers; ++l) need += 32 * T->L[kLayerLevel[l]].vox();   // dpre
    const size_t plane0 = (size_t)T->L[0].nz * T->L[0].ny * nxp_of(T->L[0].nx);
    need += 128 * plane0 + 32 * plane0;                           // Apl, Bpl
    if (need > T->cap) {
      cudaFree(T->ws);
      T->ws = nullptr;
      T->cap = 0;
      __nv_bfloat16* buf = nullptr;
      VIE_CUDA_TRY(cudaMalloc((void**)&buf, need * sizeof(__nv_bfloat16)));
      T->ws = buf;
      T->cap = need;
    }
    if (16 * V0 > T->yf_cap) {
      cudaFree(T->Yf);
      T->Yf = nullptr;
      T->yf_cap = 0;
      float* buf = nullptr;
      VIE_CUDA_TRY(cudaMalloc((void**)&buf, 16 * V0 * sizeof(float)));
      T->Yf = buf;
      T->yf_cap = 16 * V0;
    }
    __nv_bfloat16* p = T->ws;
    auto take = [&](size_t k) { __nv_bfloat16* r = p; p += k; return r; };
    T->X = take(16 * V0);
    T->dY = take(16 * V0);
    for (int l = 0; l < 4; ++l) {
      T->h[l] = take(32 * T->L[l].vox());
      T->da[l] = take(32 * T->L[l].vox());
      T->a[l] = l >= 1 ? take(32 * T->L[l].vox()) : nullptr;
    }
    for (int l = 0; l < 3; ++l) {
      T->decin[l] = take(32 * T->L[l].vox());
      T->u[l] = take(32 * T->L[l].vox());
      T->ddecin[l] = take(32 * T->L[l].vox());
    }
    for (int l = 0; l < kNumLayers; ++l) T->dpre[l] = take(32 * T->L[kLayerLevel[l]].vox());
    T->Apl = take(128 * plane0);
    T->Bpl = take(32 * plane0);
    T->plane0 = plane0;
    // rows 96..127 of A (no dx block) stay zero
    VIE_CUDA_TRY(cudaMemset(T->Apl + 96 * plane0, 0, 32 * plane0 * sizeof(__nv_bfloat16)));
    // forward maps: the inputs of enc0..enc3, dec2, dec1, dec0, out
    const __nv_bfloat16* in[kNumLayers] = {T->X, T->a[1], T->a[2], T->a[3], T->decin[2], T->decin[1], T->decin[0],
                                           T->u[0]};
    for (int l = 0; l < kNumLayers; ++l) {
      const Dims d = T->L[kLayerLevel[l]];
      tc_pick_tile(d, l <= ENC2, &T->bxf[l], &T->byf[l]);
      vie_status st = tc_encode_act(&T->mA[l], in[l], tc_cpad(kLayerDefs[l].ci), d, T->bxf[l], T->byf[l]);
      if (st != VIE_OK) return st;
      // backward data: the input is the layer's output gradient (dY for the
      // output layer, dpre[l] otherwise) with tc_cpad(co) channels
      tc_pick_tile(d, false, &T->bxb[l], &T->byb[l]);
      st = tc_encode_act(&T->mG[l], l == OUTL ? T->dY : T->dpre[l], tc_cpad(kLayerDefs[l].co), d, T->bxb[l],
                         T->byb[l]);
      if (st != VIE_OK) return st;
      const int nxp = nxp_of(d.nx);
      if ((st = tc_encode_planar(&T->mPa[l], T->Apl, 128, d, nxp, plane0)) != VIE_OK) return st;
      if ((st = tc_encode_planar(&T->mPb[l], T->Bpl, tc_cpad(kLayerDefs[l].ci), d, nxp, plane0)) != VIE_OK)
        return st;
    }
    T->n[0] = n[0];
    T->n[1] = n[1];
    T->n[2] = n[2];
  }
  // weight maps (the packed weights live in the network: encoded again
  // only when they move)
  if (T->wpack_enc == P.wpack && T->wpackf_enc == P.wpackf) return VIE_OK;
  T->wpack_enc = nullptr;
  for (int l = 0; l < kNumLayers; ++l) {
    vie_status st = tc_encode_w(&T->mW[l], P.wpack + pack_off(l), tc_cpad(kLayerDefs[l].ci), tc_npad(kLayerDefs[l].co));
    if (st != VIE_OK) return st;
    st = tc_encode_w(&T->mWf[l], P.wpackf + packf_off(l), tc_cpad(kLayerDefs[l].co), tc_npad(kLayerDefs[l].ci));
    if (st != VIE_OK) return st;
  }
  T->wpack_enc = P.wpack;
  T->wpackf_enc = P.wpackf;
  return VIE_OK;
}

static unsigned ew_grid(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

// weight and bias gradients of `layer` from its pre-activation gradient g
// (NPo channels) and its input `in` (tc_cpad(ci) channels), added to grad
static vie_status weight_grad_tc(const TcTrain* T, const TcTrainParams& P, int layer, const __nv_bfloat16* g,
                                 const __nv_bfloat16* in, cudaStream_t s) {
  const Dims d = T->L[kLayerLevel[layer]];
  const int ci = kLayerDefs[layer].ci, co = kLayerDefs[layer].co;
  const int C = tc_cpad(ci), NPo = tc_npad(co);
  const int nxp = nxp_of(d.nx);
  const int nxc = nxp / kDwChunk;
  dw_operands_kernel<<<dim3((unsigned)(2 * nxc), (unsigned)d.ny, (unsigned)d.nz), 256, 0, s>>>(
      g, NPo, co, in, C, d, nxp, nxc, T->plane0, T->Apl, T->Bpl, P.grad + layer_b_off(layer));
  VIE_LAUNCH_CHECK();
  constexpr size_t kSB32 = 128 * 128 + 9 * 32 * 128, kSB16 = 128 * 128 + 9 * 16 * 128;
  const size_t fixed = 1024 + 2 * kDwMaxStages * 8 + 64;
  const size_t SB = C == 32 ? kSB32 : kSB16;
  int stages = (int)(((size_t)T->smem_optin - fixed) / SB);
  if (stages > kDwMaxStages) stages = kDwMaxStages;
  if (stages < 2) {
    set_error("weight-gradient GEMM: %zu B per stage does not fit", SB);
    return VIE_ERR_INVALID;
  }
  const size_t smem = fixed + (size_t)stages * SB;
  DwArgs a{};
  a.d = d;
  a.nxc = nxp / kDwChunk;
  a.stages = stages;
  a.partial = T->partial;
  a.bad = P.bad;
  // at least kDwMinChunks chunks per CTA where the level is small: fewer
  // partial sums to write and reduce
  const long nchunks = (long)d.nz * d.ny * a.nxc;
  long want = (nchunks + kDwMinChunks - 1) / kDwMinChunks;
  if (want < 1) want = 1;
  const int nb = (int)(want < T->sms ? want : T->sms);
  if (C == 32) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(dw_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dw_tc_kernel<32><<<nb, kDwThreads, smem, s>>>(T->mPa[layer], T->mPb[layer], a);
  } else {
    VIE_CUDA_TRY(cudaFuncSetAttribute(dw_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dw_tc_kernel<16><<<nb, kDwThreads, smem, s>>>(T->mPa[layer], T->mPb[layer], a);
  }
  VIE_LAUNCH_CHECK();
  const int nred = 27 * 32 * C, slices = nb < 16 ? nb : 16;
  dw_reduce_kernel<<<dim3((unsigned)((nred + 255) / 256), (unsigned)slices), 256, 0, s>>>(
      T->partial, nb, C, ci, co, P.grad + layer_w_off(layer));
  VIE_LAUNCH_CHECK();
  return VIE_OK;
}

vie_status tc_train_accumulate(TcTrain** pt, const TcTrainParams& P, const int n[3], const double2* chi,
                               const float2* r, const float2* e, double* loss, cudaStream_t s) {
  vie_status st = tc_train_prepare(pt, P, n);
  if (st != VIE_OK) return st;
  TcTrain* T = *pt;
  const Dims L0 = T->L[0];
  const size_t V0 = L0.vox();
  // ---- forward ----
  if ((st = tc_pack_input<float2>(r, chi, L0, T->norm, T->X, s)) != VIE_OK) return st;
  const double* ssr = T->norm + kTcNormBlocks;
  auto fwd = [&](int layer, int mode, __nv_bfloat16* out, __nv_bfloat16* out2, int level2,
                 const __nv_bfloat16* skip, float* outf) {
    TcConvArgs a{};
    a.d = T->L[kLayerLevel[layer]];
    a.d2 = level2 >= 0 ? T->L[level2] : a.d;
    a.bx = T->bxf[layer];
    a.by = T->byf[layer];
    a.bias = P.master + layer_b_off(layer);
    a.co = kLayerDefs[layer].co;
    a.out = out;
    a.out2 = out2;
    a.skip = skip;
    a.outf = outf;
    a.bad = P.bad;
    return tc_conv(T->mA[layer], T->mW[layer], tc_cpad(kLayerDefs[layer].ci), tc_npad(kLayerDefs[layer].co), mode, a,
                   s);
  };
  for (int l = 0; l < 3; ++l)
    if ((st = fwd(ENC0 + l, TC_RELU_POOL, T->h[l], T->a[l + 1], l + 1, nullptr, nullptr)) != VIE_OK) return st;
  if ((st = fwd(ENC3, TC_RELU_UPADD, T->h[3], T->decin[2], 2, T->h[2], nullptr)) != VIE_OK) return st;
  if ((st = fwd(DEC2, TC_RELU_UPADD, T->u[2], T->decin[1], 1, T->h[1], nullptr)) != VIE_OK) return st;
  if ((st = fwd(DEC1, TC_RELU_UPADD, T->u[1], T->decin[0], 0, T->h[0], nullptr)) != VIE_OK) return st;
  if ((st = fwd(DEC0, TC_RELU_BF16, T->u[0], nullptr, -1, nullptr, nullptr)) != VIE_OK) return st;
  if ((st = fwd(OUTL, TC_LINEAR_F32, nullptr, nullptr, -1, nullptr, T->Yf)) != VIE_OK) return st;
  // ---- loss ----
  double* sums = T->norm + kTcNormBlocks + 1;
  VIE_CUDA_TRY(cudaMemsetAsync(sums, 0, 2 * sizeof(double), s));
  loss_cl_kernel<<<ew_grid(V0), 256, 0, s>>>(T->Yf, e, r, V0, ssr, sums);
  loss_grad_cl_kernel<<<ew_grid(V0), 256, 0, s>>>(T->Yf, e, r, V0, ssr, sums, T->dY);
  VIE_LAUNCH_CHECK();
  // ---- backward ----
  auto bwd = [&](int layer, __nv_bfloat16* out, const __nv_bfloat16* mask) {
    TcConvArgs a{};
    a.d = T->L[kLayerLevel[layer]];
    a.d2 = a.d;
    a.bx = T->bxb[layer];
    a.by = T->byb[layer];
    a.out = out;
    a.skip = mask;
    a.bad = P.bad;
    return tc_conv(T->mG[layer], T->mWf[layer], tc_cpad(kLayerDefs[layer].co), tc_npad(kLayerDefs[layer].ci),
                   TC_GRAD_BF16, a, s);
  };
  const Dims* L = T->L;
  // output layer: input u_0 = relu(dec0)
  if ((st = weight_grad_tc(T, P, OUTL, T->dY, T->u[0], s)) != VIE_OK) return st;
  if ((st = bwd(OUTL, T->dpre[DEC0], T->u[0])) != VIE_OK) return st;
  // decoders: input decin_l = up(u_{l+1}) + h_l (u_3 = h_3)
  for (int l = 0; l <= 2; ++l) {
    const int layer = DEC0 - l;   // dec0, dec1, dec2
    if ((st = weight_grad_tc(T, P, layer, T->dpre[layer], T->decin[l], s)) != VIE_OK) return st;
    if ((st = bwd(layer, T->ddecin[l], nullptr)) != VIE_OK) return st;
    const int coarse_layer = l == 2 ? ENC3 : layer - 1;      // producer of the coarse tensor
    const __nv_bfloat16* coarse = l == 2 ? T->h[3] : T->u[l + 1];
    upback_mask_kernel<<<ew_grid(L[l + 1].vox() * 4), 256, 0, s>>>(T->ddecin[l], L[l], coarse, L[l + 1],
                                                                    T->dpre[coarse_layer]);
    VIE_LAUNCH_CHECK();
  }
  // encoders: input a_l = pool(h_{l-1}) (X for enc0); h_{l-1} also feeds decin_{l-1}
  for (int l = 3; l >= 0; --l) {
    const int layer = ENC0 + l;
    const __nv_bfloat16* in = l == 0 ? T->X : T->a[l];
    if ((st = weight_grad_tc(T, P, layer, T->dpre[layer], in, s)) != VIE_OK) return st;
    if (l == 0) break;
    if ((st = bwd(layer, T->da[l], nullptr)) != VIE_OK) return st;
    poolback_mask_kernel<<<ew_grid(L[l - 1].vox() * 4), 256, 0, s>>>(T->ddecin[l - 1], T->da[l], L[l], T->h[l - 1],
                                                                      L[l - 1], T->dpre[ENC0 + l - 1]);
    VIE_LAUNCH_CHECK();
  }
  if (loss) {
    double h[3] = {0, 0, 0};
    VIE_CUDA_TRY(cudaMemcpyAsync(h, sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA_TRY(cudaStreamSynchronize(s));
    *loss = h[1] > 0 ? h[0] / h[1] : 0.0;
  }
  return VIE_OK;
}

}  // namespace vie
