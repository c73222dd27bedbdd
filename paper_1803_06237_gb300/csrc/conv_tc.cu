// Tensor-core inference path of the learned preconditioner.
//
// Activations are channels-last BF16, [z][y][x][C] with C = 16 (network
// input, 8 channels used) or 32.  A 3x3x3 convolution with zero padding is
// an implicit GEMM: M = 128 output voxels (a bx x by patch of one z plane),
// N = 16 or 32 output channels, K = 27 taps x C input channels, FP32
// accumulation in tensor memory.
//
// One persistent CTA (two per SM) runs three roles:
//   warp 0   TMA producer: the 27 weight taps once, then per tile and per
//            (dz, dx) one box of (by + 2) rows x bx voxels x C channels at
//            (x0 + dx - 1, y0 - 1, z + dz - 1); the TMA unit zero-fills the
//            padding outside the grid;
//   warp 1   tcgen05.mma issuer: per box three taps (dy = 0, 1, 2 are the
//            same box shifted by bx rows, a multiple of the swizzle atom),
//            C / 16 MMAs of 128 x N x 16 each, into one of two TMEM
//            accumulators;
//   warps 2-5 epilogue: tcgen05.ld of the accumulator (warp w owns TMEM lanes
//            32 (w % 4) ..), bias, ReLU and BF16 store, or the fused output
//            step z = v + Net(v) / s of the preconditioner.
// Stages are handed over with mbarriers (TMA transaction counts,
// tcgen05.commit); every wait is bounded and a timeout is reported in *bad.
//
// Every kernel of the inference chain is launched with programmatic stream
// serialisation: it lets its dependents launch at entry, sets up barriers
// and tensor memory and prefetches the (immutable) weights, and only then
// waits (griddepcontrol.wait) for the kernel that produced its input.
#include <stdio.h>

#include <type_traits>

#include "net.cuh"
#include "tc.cuh"

namespace vie {

constexpr int kTcMaxStages = 8;
constexpr int kTcThreads = 192;

template <int C, int N, int MODE>
__global__ void __launch_bounds__(kTcThreads, 2) conv_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmW,
                                                                 const TcConvArgs a) {
  constexpr int ROWB = C * 2;                        // bytes per voxel row / weight row
  constexpr uint32_t WTAP = (uint32_t)N * ROWB;      // bytes of one weight tap
  constexpr uint32_t NCOLS = 2 * N < 32 ? 32 : 2 * N;
  constexpr int KSTEPS = C / 16;
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, N);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sW = base;
  unsigned char* sA = base + 27 * WTAP;
  const int bx = a.bx, by = a.by;
  const uint32_t S = (uint32_t)a.stages;
  const uint32_t stage_bytes = (uint32_t)((by + 2) * bx * ROWB);
  uint64_t* full = (uint64_t*)(sA + S * stage_bytes);
  uint64_t* empty = full + kTcMaxStages;
  uint64_t* wbar = empty + kTcMaxStages;
  uint64_t* tfull = wbar + 1;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_x = (a.d.nx + bx - 1) / bx, tiles_y = (a.d.ny + by - 1) / by;
  const int ntiles = tiles_x * tiles_y * a.d.nz;

  pdl_launch_dependents();
  if (threadIdx.x == 0) {
    for (uint32_t i = 0; i < S; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(wbar, 1);
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&tfull[i], 1);
      tc::mbar_init(&tempty[i], 128);
    }
    tc::mbar_init(drain, 1);
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
    tc::prefetch_tensormap(&tmW);
    tc::mbar_arrive_expect_tx(wbar, 27 * WTAP);
    for (int t = 0; t < 27; ++t) tc::tma_load_3d(sW + t * WTAP, &tmW, wbar, 0, 0, t);
    pdl_wait();                     // the producer of the input activation has completed
    uint32_t it = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x) {
      const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, z = tile / (tiles_x * tiles_y);
      for (int s9 = 0; s9 < 9; ++s9, ++it) {
        const int dz = s9 / 3, dx = s9 % 3;
        const uint32_t stage = it % S, round = it / S;
        if (!tc::mbar_wait(&empty[stage], (round & 1) ^ 1, abort)) break;
        tc::mbar_arrive_expect_tx(&full[stage], stage_bytes);
        tc::tma_load_4d(sA + stage * stage_bytes, &tmA, &full[stage], 0, tx * bx + dx - 1, ty * by - 1,
                        z + dz - 1);
      }
    }
    if (*abort) {
      // let the copies already issued land before the CTA exits
      for (uint32_t k = 0; k < S && k < it; ++k) {
        const uint32_t last = it - 1 - k;
        volatile int never = 0;
        tc::mbar_wait(&full[last % S], (last / S) & 1, &never);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    bool issued = false;
    if (tc::mbar_wait(wbar, 0, abort)) {
      const uint32_t sWa = tc::smem_u32(sW), sAa = tc::smem_u32(sA);
      uint32_t it = 0, local = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x, ++local) {
        const uint32_t b = local & 1, use = local >> 1;
        if (!tc::mbar_wait(&tempty[b], (use & 1) ^ 1, abort)) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + b * N;
        bool ok = true;
        for (int s9 = 0; s9 < 9; ++s9, ++it) {
          const int dz = s9 / 3, dx = s9 % 3;
          const uint32_t stage = it % S, round = it / S;
          if (!tc::mbar_wait(&full[stage], round & 1, abort)) { ok = false; break; }
          tc::fence_after_sync();
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            const int tap = (dz * 3 + dy) * 3 + dx;
            const uint32_t aa = sAa + stage * stage_bytes + (uint32_t)(dy * bx * ROWB);
            const uint32_t ba = sWa + (uint32_t)tap * WTAP;
#pragma unroll
            for (int k = 0; k < KSTEPS; ++k)
              tc::mma_bf16(d, tc::smem_desc(aa + 32 * k, ROWB), tc::smem_desc(ba + 32 * k, ROWB), IDESC,
                           (s9 | dy | k) != 0);
          }
          issued = true;
          tc::mma_commit(&empty[stage]);    // frees the stage when these MMAs are done
        }
        if (!ok) break;
        tc::mma_commit(&tfull[b]);          // accumulator b is complete
      }
    }
    if (*abort && issued) {
      tc::mma_commit(drain);
      volatile int never = 0;
      tc::mbar_wait(drain, 0, &never);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    pdl_wait();                     // writes and the input scale come after the producer
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const int xl = row % bx, yl = row / bx;
    float bias[N];
#pragma unroll
    for (int o = 0; o < N; ++o) bias[o] = o < a.co ? __ldg(a.bias + o) : 0.f;
    double inv = 0.0;
    if (MODE != TC_RELU_BF16) {
      const double ss = *a.sumsq;
      inv = ss > 0.0 ? sqrt(ss / (3.0 * (double)a.d.vox())) : 0.0;
    }
    uint32_t local = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x, ++local) {
      const uint32_t b = local & 1, use = local >> 1;
      // every lane waits; the vote also reconverges the warp for the
      // warp-wide (.sync.aligned) tensor-memory load
      const bool ok = tc::mbar_wait(&tfull[b], use & 1, abort);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc::fence_after_sync();
      float acc[N];
      if constexpr (N == 32) tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + b * N, acc);
      else tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + b * N, acc);
      tc::fence_before_sync();
      tc::mbar_arrive(&tempty[b]);
      const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, z = tile / (tiles_x * tiles_y);
      const int x = tx * bx + xl, y = ty * by + yl;
      if (x >= a.d.nx || y >= a.d.ny) continue;
      const size_t vox = ((size_t)z * a.d.ny + y) * a.d.nx + x;
      if constexpr (MODE == TC_RELU_BF16) {
        uint4 pk[N / 8];
        uint32_t* w = (uint32_t*)pk;
#pragma unroll
        for (int o = 0; o < N; o += 2) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(fmaxf(acc[o] + bias[o], 0.f),
                                                          fmaxf(acc[o + 1] + bias[o + 1], 0.f));
          w[o / 2] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        uint4* dst = reinterpret_cast<uint4*>(a.out + vox * N);
#pragma unroll
        for (int i = 0; i < N / 8; ++i) dst[i] = pk[i];
      } else {
        using V = typename std::conditional<MODE == TC_UNPACK_C64, float2, double2>::type;
        const V* v = (const V*)a.v;
        V* zo = (V*)a.z;
        const size_t V0 = a.d.vox();
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double re = (double)(acc[c] + bias[c]) * inv, im = (double)(acc[3 + c] + bias[3 + c]) * inv;
          V vi = v[(size_t)c * V0 + vox];
          if (isfinite(re) && isfinite(im)) {
            vi.x += re;
            vi.y += im;
          } else {
            atomicExch(a.bad, 1);
          }
          zo[(size_t)c * V0 + vox] = vi;
        }
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

void tc_pick_tile(Dims d, int* bx, int* by) {
  static const int cand[4][2] = {{16, 8}, {32, 4}, {64, 2}, {128, 1}};
  double best = 1e300;
  for (auto& c : cand) {
    const double px = (double)((d.nx + c[0] - 1) / c[0]) * c[0];
    const double py = (double)((d.ny + c[1] - 1) / c[1]) * c[1];
    const double cost = px * py * (c[1] + 2) / c[1];
    if (cost < best) {
      best = cost;
      *bx = c[0];
      *by = c[1];
    }
  }
}

static vie_status encode(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                         const cuuint64_t* strides, const cuuint32_t* box, int C) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return VIE_ERR_CUDA;
  }
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        C == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return VIE_ERR_CUDA;
  }
  return VIE_OK;
}

vie_status tc_encode_act(CUtensorMap* map, const __nv_bfloat16* base, int C, Dims d, int bx, int by) {
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * d.nx, (cuuint64_t)C * 2 * d.nx * d.ny};
  const cuuint32_t box[4] = {(cuuint32_t)C, (cuuint32_t)bx, (cuuint32_t)(by + 2), 1};
  return encode(map, base, 4, dims, strides, box, C);
}

vie_status tc_encode_w(CUtensorMap* map, const __nv_bfloat16* w, int C, int N) {
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)N, 27};
  const cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * N};
  const cuuint32_t box[3] = {(cuuint32_t)C, (cuuint32_t)N, 1};
  return encode(map, w, 3, dims, strides, box, C);
}

struct DevInfo {
  int sms = 0;
  int smem_sm = 0;        // shared memory per SM (bytes)
  int smem_reserved = 0;  // reserved by the system per block
};

static const DevInfo& dev_info() {
  static DevInfo d;
  if (!d.sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&d.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&d.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return d;
}

constexpr size_t kTcBarrierBytes = 32 * sizeof(uint64_t);

// Stages and resident CTAs per SM for a tile: two CTAs per SM with the
// deepest ring that still fits (at least three stages), else one CTA with
// up to kTcMaxStages stages.
static void plan_stages(size_t fixed, size_t stage, const DevInfo& d, int* stages, int* per_sm) {
  const size_t sm = (size_t)d.smem_sm, rsv = (size_t)d.smem_reserved;
  for (int s = kTcMaxStages; s >= 3; --s)
    if (2 * (fixed + s * stage + rsv) <= sm) {
      *stages = s;
      *per_sm = 2;
      return;
    }
  for (int s = kTcMaxStages; s >= 2; --s)
    if (fixed + s * stage + rsv <= sm) {
      *stages = s;
      *per_sm = 1;
      return;
    }
  *stages = 0;
  *per_sm = 0;
}

template <int C, int N, int MODE>
static vie_status launch_conv(const CUtensorMap& A, const CUtensorMap& W, TcConvArgs args, cudaStream_t s) {
  static bool configured = false;
  auto kern = conv_tc_kernel<C, N, MODE>;
  const DevInfo& dv = dev_info();
  const size_t fixed = 1024 + 27 * (size_t)N * C * 2 + kTcBarrierBytes;
  if (!configured) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      dv.smem_sm - dv.smem_reserved));
    VIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    configured = true;
  }
  const size_t stage = (size_t)(args.by + 2) * args.bx * C * 2;
  int stages = 0, per_sm = 0;
  plan_stages(fixed, stage, dv, &stages, &per_sm);
  if (per_sm < 1 || dv.sms < 1) {
    set_error("tensor-core convolution does not fit on an SM (%zu B per stage)", stage);
    return VIE_ERR_INVALID;
  }
  args.stages = stages;
  const size_t smem = fixed + (size_t)stages * stage;
  const Dims d = args.d;
  const long ntiles = (long)((d.nx + args.bx - 1) / args.bx) * ((d.ny + args.by - 1) / args.by) * d.nz;
  long grid = (long)dv.sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return VIE_OK;
  VIE_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(kTcThreads), smem, s, A, W, args));
  return VIE_OK;
}

vie_status tc_conv(const CUtensorMap& A, const CUtensorMap& W, int C, int N, int mode, const TcConvArgs& args,
                   cudaStream_t s) {
  if (args.bx * args.by != 128 || args.bx % 8 != 0) {
    set_error("tensor-core convolution: tile %d x %d is not 128 voxels", args.bx, args.by);
    return VIE_ERR_INVALID;
  }
  if (C == 16 && N == 32 && mode == TC_RELU_BF16) return launch_conv<16, 32, TC_RELU_BF16>(A, W, args, s);
  if (C == 32 && N == 32 && mode == TC_RELU_BF16) return launch_conv<32, 32, TC_RELU_BF16>(A, W, args, s);
  if (C == 32 && N == 16 && mode == TC_UNPACK_C64) return launch_conv<32, 16, TC_UNPACK_C64>(A, W, args, s);
  if (C == 32 && N == 16 && mode == TC_UNPACK_C128) return launch_conv<32, 16, TC_UNPACK_C128>(A, W, args, s);
  set_error("no tensor-core convolution for C=%d N=%d mode=%d", C, N, mode);
  return VIE_ERR_INVALID;
}

// ---------------------------------------------------------------------------
// channels-last BF16 element-wise steps
// ---------------------------------------------------------------------------
static unsigned grid_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

// sum |v|^2 over the 3 V entries as kTcNormBlocks partial sums (no atomics)
template <typename V>
__global__ void __launch_bounds__(256) sumsq_partial_kernel(const V* __restrict__ v, size_t n,
                                                            double* __restrict__ part) {
  pdl_launch_dependents();
  pdl_wait();
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const V a = v[i];
    acc += (double)a.x * a.x + (double)a.y * a.y;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// X[vox][16]: re v_c s (c = 0..2), im v_c s, re chi, im chi, 8 zeros;
// s = sqrt(3 V / sum|v|^2).  Every block totals the partial sums; block 0
// also stores the total in part[kTcNormBlocks] for the output step.
template <typename V>
__global__ void __launch_bounds__(256) pack_cl_kernel(const V* __restrict__ v, const double2* __restrict__ chi,
                                                      size_t vox, double* __restrict__ part,
                                                      __nv_bfloat16* __restrict__ X) {
  pdl_launch_dependents();
  pdl_wait();
  __shared__ double tot;
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = threadIdx.x; i < kTcNormBlocks; i += 32) t += part[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) {
      tot = t;
      if (blockIdx.x == 0) part[kTcNormBlocks] = t;
    }
  }
  __syncthreads();
  const double ss = tot;
  const float s = ss > 0.0 ? (float)sqrt(3.0 * (double)vox / ss) : 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < vox; i += (size_t)gridDim.x * blockDim.x) {
    float f[8];
    for (int c = 0; c < 3; ++c) {
      const V a = v[(size_t)c * vox + i];
      f[c] = (float)a.x * s;
      f[3 + c] = (float)a.y * s;
    }
    f[6] = (float)chi[i].x;
    f[7] = (float)chi[i].y;
    uint4 lo, hi = make_uint4(0, 0, 0, 0);
    uint32_t* w = (uint32_t*)&lo;
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
      w[k] = *reinterpret_cast<const uint32_t*>(&h2);
    }
    uint4* dst = reinterpret_cast<uint4*>(X + i * 16);
    dst[0] = lo;
    dst[1] = hi;
  }
}

__device__ __forceinline__ void bf8_to_f(uint4 u, float (&f)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 t = __bfloat1622float2(h[k]);
    f[2 * k] = t.x;
    f[2 * k + 1] = t.y;
  }
}
__device__ __forceinline__ uint4 f_to_bf8(const float (&f)[8]) {
  uint4 u;
  uint32_t* w = (uint32_t*)&u;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    w[k] = *reinterpret_cast<const uint32_t*>(&h2);
  }
  return u;
}

// average over the 2 x 2 (y, x) fine voxels that exist; one thread per
// (coarse voxel, group of 8 channels), 32 channels
__global__ void pool_cl_kernel(const __nv_bfloat16* __restrict__ in, Dims f, __nv_bfloat16* __restrict__ out,
                               Dims c) {
  pdl_launch_dependents();
  pdl_wait();
  const size_t n = c.vox() * 4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i & 3);
    const size_t cv = i >> 2;
    const int x = (int)(cv % c.nx), y = (int)((cv / c.nx) % c.ny), z = (int)(cv / ((size_t)c.nx * c.ny));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int cnt = 0;
    for (int oy = 0; oy < 2; ++oy)
      for (int ox = 0; ox < 2; ++ox) {
        const int yy = 2 * y + oy, xx = 2 * x + ox;
        if (yy >= f.ny || xx >= f.nx) continue;
        float t[8];
        bf8_to_f(*reinterpret_cast<const uint4*>(in + (((size_t)z * f.ny + yy) * f.nx + xx) * 32 + 8 * g), t);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += t[k];
        ++cnt;
      }
    const float r = 1.f / (float)cnt;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] *= r;
    *reinterpret_cast<uint4*>(out + cv * 32 + 8 * g) = f_to_bf8(acc);
  }
}

// out = up(coarse) + skip (nearest neighbour in y and x), 32 channels
__global__ void up_add_cl_kernel(const __nv_bfloat16* __restrict__ coarse, Dims c,
                                 const __nv_bfloat16* __restrict__ skip, __nv_bfloat16* __restrict__ out, Dims f) {
  pdl_launch_dependents();
  pdl_wait();
  const size_t n = f.vox() * 4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i & 3);
    const size_t fv = i >> 2;
    const int x = (int)(fv % f.nx), y = (int)((fv / f.nx) % f.ny), z = (int)(fv / ((size_t)f.nx * f.ny));
    float a[8], b[8];
    bf8_to_f(*reinterpret_cast<const uint4*>(coarse + (((size_t)z * c.ny + y / 2) * c.nx + x / 2) * 32 + 8 * g), a);
    bf8_to_f(*reinterpret_cast<const uint4*>(skip + fv * 32 + 8 * g), b);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] += b[k];
    *reinterpret_cast<uint4*>(out + fv * 32 + 8 * g) = f_to_bf8(a);
  }
}

template <typename V>
vie_status tc_pack_input(const V* v, const double2* chi, Dims d, double* part, __nv_bfloat16* X, cudaStream_t s) {
  VIE_CUDA_TRY(launch_pdl(sumsq_partial_kernel<V>, dim3(kTcNormBlocks), dim3(256), 0, s, v, 3 * d.vox(), part));
  VIE_CUDA_TRY(launch_pdl(pack_cl_kernel<V>, dim3(grid_for(d.vox())), dim3(256), 0, s, v, chi, d.vox(), part, X));
  return VIE_OK;
}
template vie_status tc_pack_input<float2>(const float2*, const double2*, Dims, double*, __nv_bfloat16*, cudaStream_t);
template vie_status tc_pack_input<double2>(const double2*, const double2*, Dims, double*, __nv_bfloat16*,
                                           cudaStream_t);

vie_status tc_pool(const __nv_bfloat16* in, Dims f, __nv_bfloat16* out, Dims c, cudaStream_t s) {
  VIE_CUDA_TRY(launch_pdl(pool_cl_kernel, dim3(grid_for(c.vox() * 4)), dim3(256), 0, s, in, f, out, c));
  return VIE_OK;
}

vie_status tc_up_add(const __nv_bfloat16* coarse, Dims c, const __nv_bfloat16* skip, __nv_bfloat16* out, Dims f,
                     cudaStream_t s) {
  VIE_CUDA_TRY(launch_pdl(up_add_cl_kernel, dim3(grid_for(f.vox() * 4)), dim3(256), 0, s, coarse, c, skip, out, f));
  return VIE_OK;
}

}  // namespace vie
