// Tensor-core inference path of the learned preconditioner.
//
// Activations are channels-last BF16, [z][y][x][C] with C = 16 (network
// input, 8 channels used) or 32.  A 3x3x3 convolution with zero padding is
// an implicit GEMM on the tcgen05 tensor cores with FP32 accumulation in
// tensor memory:
//   M = 128 input positions of a tile: bx columns in x (the bx - 2 output
//       columns and a one-voxel halo on each side) times by rows in y, one
//       z plane;
//   N = 3 x NP: for every dx tap the NP (16 or 32, padded) output channels,
//       so that one A tile feeds the three dx taps at once;
//   K = 9 (dz, dy) taps x C channels, C / 16 MMAs of 128 x N x 16 per tap.
// Row m of the accumulator then holds, for input position p(m), the partial
// sums D[p][dx][o] = sum over (dz, dy, c) of X[p + (dz, dy) - 1][c] W[dz][dy][dx][o][c];
// output voxel x is D[x - 1][0] + D[x][1] + D[x + 1][2], which the epilogue
// forms with two warp shuffles (the x neighbours of a row are the adjacent
// lanes of the same warp).
//
// One persistent CTA (two per SM) runs three roles:
//   warp 0   TMA producer: the 27 weight taps once, then per tile and per
//            dz one box of (by + 2) rows x bx columns x C channels at
//            (x0 - 1, y0 - 1, z + dz - 1); the TMA unit zero-fills the
//            padding outside the grid;
//   warp 1   tcgen05.mma issuer: per box the three dy taps (the same box
//            shifted by bx rows, a multiple of the swizzle atom) into one of
//            two TMEM accumulators;
//   warps 2-5 epilogue: tcgen05.ld of the accumulator (warp w owns TMEM
//            lanes 32 (w % 4) ..), the dx shift-add, bias and ReLU, then one
//            of: a BF16 store; a store plus the 2 x 2 average pooling of the
//            next level; the nearest upsampling added to the finer level's
//            skip tensor; or the output step z = v + Net(v) / s.
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

constexpr int kTcMaxStages = 16;
constexpr int kTcThreads = 192;

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <int NP>
__device__ __forceinline__ void tmem_ld_np(uint32_t taddr, float (&v)[NP]) {
  if constexpr (NP == 32) tc::tmem_ld32(taddr, v);
  else tc::tmem_ld16(taddr, v);
}

template <int NP>
__device__ __forceinline__ void store_bf16_row(__nv_bfloat16* dst, const float (&v)[NP]) {
  uint4 pk[NP / 8];
  uint32_t* w = (uint32_t*)pk;
#pragma unroll
  for (int o = 0; o < NP; o += 2) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[o], v[o + 1]);
    w[o / 2] = *reinterpret_cast<const uint32_t*>(&h2);
  }
  uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int i = 0; i < NP / 8; ++i) d[i] = pk[i];
}

template <int C, int NP, int MODE>
__global__ void __launch_bounds__(kTcThreads, 2) conv_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmW,
                                                                 const TcConvArgs a) {
  constexpr int ROWB = C * 2;                        // bytes per voxel row / weight row
  constexpr int N = 3 * NP;                          // MMA N: NP output channels for each dx tap
  constexpr uint32_t WTAP = (uint32_t)NP * ROWB;     // bytes of one weight tap
  constexpr uint32_t NCOLS = 2 * N <= 128 ? 128 : 256;
  constexpr int KSTEPS = C / 16;
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, N);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sW = base;
  unsigned char* sA = base + 27 * WTAP;
  const int bx = a.bx, bxo = a.bx - 2, by = a.by;
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
  const int tiles_x = (a.d.nx + bxo - 1) / bxo, tiles_y = (a.d.ny + by - 1) / by;
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
      for (int dz = 0; dz < 3; ++dz, ++it) {
        const uint32_t stage = it % S, round = it / S;
        if (!tc::mbar_wait(&empty[stage], (round & 1) ^ 1, abort)) break;
        tc::mbar_arrive_expect_tx(&full[stage], stage_bytes);
        tc::tma_load_4d(sA + stage * stage_bytes, &tmA, &full[stage], 0, tx * bxo - 1, ty * by - 1, z + dz - 1);
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
      // descriptors of the first weight tap and of ring stage 0; every MMA
      // adds its byte offset to the start-address field
      const uint64_t dW0 = tc::smem_desc(tc::smem_u32(sW), ROWB), dA0 = tc::smem_desc(tc::smem_u32(sA), ROWB);
      uint32_t it = 0, local = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x, ++local) {
        const uint32_t b = local & 1, use = local >> 1;
        if (!tc::mbar_wait(&tempty[b], (use & 1) ^ 1, abort)) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + b * N;
        bool ok = true;
        for (int dz = 0; dz < 3; ++dz, ++it) {
          const uint32_t stage = it % S, round = it / S;
          if (!tc::mbar_wait(&full[stage], round & 1, abort)) { ok = false; break; }
          const uint64_t dA = tc::desc_add(dA0, stage * stage_bytes);
          const uint32_t row_step = (uint32_t)(bx * ROWB);
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            // B rows (dx, o) of taps (dz, dy, 0..2) are consecutive in the packed weights
            const uint64_t a_dy = tc::desc_add(dA, dy * row_step);
            const uint64_t b_dy = tc::desc_add(dW0, (uint32_t)((dz * 3 + dy) * 3) * WTAP);
#pragma unroll
            for (int k = 0; k < KSTEPS; ++k)
              tc::mma_bf16(d, tc::desc_add(a_dy, 32 * k), tc::desc_add(b_dy, 32 * k), IDESC, (dz | dy | k) != 0);
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
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    float bias[NP];
#pragma unroll
    for (int o = 0; o < NP; ++o) bias[o] = (a.bias && o < a.co) ? __ldg(a.bias + o) : 0.f;
    double inv = 0.0;
    if constexpr (MODE == TC_UNPACK_C64 || MODE == TC_UNPACK_C128) {
      const double ss = *a.sumsq;
      inv = ss > 0.0 ? sqrt(ss / (3.0 * (double)a.d.vox())) : 0.0;
    }
    uint32_t local = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++local) {
      // the abort flag is read once per warp so that all lanes leave together
      if (__shfl_sync(0xffffffffu, (int)*abort, 0)) break;
      const uint32_t b = local & 1, use = local >> 1;
      // every lane waits; the vote also reconverges the warp for the
      // warp-wide (.sync.aligned) tensor-memory loads and the shuffles
      const bool ok = tc::mbar_wait(&tfull[b], use & 1, abort);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc::fence_after_sync();
      const uint32_t t0 = tmem + lane_base + b * N;
      float acc[NP], t[NP];
      tmem_ld_np<NP>(t0 + NP, acc);                 // dx = 1: this position
      tmem_ld_np<NP>(t0, t);                        // dx = 0: taken from position x - 1
#pragma unroll
      for (int o = 0; o < NP; ++o) acc[o] += __shfl_up_sync(0xffffffffu, t[o], 1);
      tmem_ld_np<NP>(t0 + 2 * NP, t);               // dx = 2: taken from position x + 1
#pragma unroll
      for (int o = 0; o < NP; ++o) acc[o] += __shfl_down_sync(0xffffffffu, t[o], 1);
      tc::fence_before_sync();
      tc::mbar_arrive(&tempty[b]);
      // lanes at xl = 0 and xl = bx - 1 are the halo: their neighbours lie in
      // another row of the tile, and they produce no output
      const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, z = tile / (tiles_x * tiles_y);
      const int x = tx * bxo + xl - 1, y = ty * by + yl;
      const bool valid = xl >= 1 && xl <= bx - 2 && x < a.d.nx && y < a.d.ny;
      const size_t vox = valid ? ((size_t)z * a.d.ny + y) * a.d.nx + x : 0;
      if constexpr (MODE == TC_RELU_BF16) {
        if (valid) {
          float h[NP];
#pragma unroll
          for (int o = 0; o < NP; ++o) h[o] = fmaxf(acc[o] + bias[o], 0.f);
          store_bf16_row<NP>(a.out + vox * NP, h);
        }
      } else if constexpr (MODE == TC_RELU_POOL) {
        // bx = 16: the block (x, x + 1) x (y, y + 1) with x and y even is
        // lanes (l, l + 1, l + 16, l + 17) of this warp, l with xl odd and
        // l < 16; the average is taken over the stored (BF16) values that exist
        float h[NP];
#pragma unroll
        for (int o = 0; o < NP; ++o) h[o] = valid ? bf16_round(fmaxf(acc[o] + bias[o], 0.f)) : 0.f;
        if (valid) store_bf16_row<NP>(a.out + vox * NP, h);
        float cnt = valid ? 1.f : 0.f;
#pragma unroll
        for (int o = 0; o < NP; ++o) h[o] += __shfl_down_sync(0xffffffffu, h[o], 1);
        cnt += __shfl_down_sync(0xffffffffu, cnt, 1);
#pragma unroll
        for (int o = 0; o < NP; ++o) h[o] += __shfl_down_sync(0xffffffffu, h[o], 16);
        cnt += __shfl_down_sync(0xffffffffu, cnt, 16);
        if (valid && (xl & 1) && lane < 16) {
          const float r = 1.f / cnt;                // cnt is 1, 2 or 4: exact
#pragma unroll
          for (int o = 0; o < NP; ++o) h[o] *= r;
          const size_t cv = ((size_t)z * a.d2.ny + (y >> 1)) * a.d2.nx + (x >> 1);
          store_bf16_row<NP>(a.out2 + cv * NP, h);
        }
      } else if constexpr (MODE == TC_RELU_UPADD) {
        if (valid) {
          float u[NP];
#pragma unroll
          for (int o = 0; o < NP; ++o) u[o] = bf16_round(fmaxf(acc[o] + bias[o], 0.f));
          if (a.out) store_bf16_row<NP>(a.out + vox * NP, u);
          for (int oy = 0; oy < 2; ++oy) {
            const int fy = 2 * y + oy;
            if (fy >= a.d2.ny) continue;
            for (int ox = 0; ox < 2; ++ox) {
              const int fx = 2 * x + ox;
              if (fx >= a.d2.nx) continue;
              const size_t fv = ((size_t)z * a.d2.ny + fy) * a.d2.nx + fx;
              const uint4* sk = reinterpret_cast<const uint4*>(a.skip + fv * NP);
              float o8[NP];
#pragma unroll
              for (int i = 0; i < NP / 8; ++i) {
                const uint4 w = sk[i];
                const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  const float2 f = __bfloat1622float2(h2[k]);
                  o8[8 * i + 2 * k] = u[8 * i + 2 * k] + f.x;
                  o8[8 * i + 2 * k + 1] = u[8 * i + 2 * k + 1] + f.y;
                }
              }
              store_bf16_row<NP>(a.out2 + fv * NP, o8);
            }
          }
        }
      } else if constexpr (MODE == TC_LINEAR_F32) {
        if (valid) {
          float4* d = reinterpret_cast<float4*>(a.outf + vox * NP);
#pragma unroll
          for (int i = 0; i < NP / 4; ++i)
            d[i] = make_float4(acc[4 * i] + bias[4 * i], acc[4 * i + 1] + bias[4 * i + 1],
                               acc[4 * i + 2] + bias[4 * i + 2], acc[4 * i + 3] + bias[4 * i + 3]);
        }
      } else if constexpr (MODE == TC_GRAD_BF16) {
        if (valid) {
          if (a.skip) {
            const uint4* mk = reinterpret_cast<const uint4*>(a.skip + vox * NP);
#pragma unroll
            for (int i = 0; i < NP / 8; ++i) {
              const uint4 w = mk[i];
              const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(h2[k]);
                if (!(f.x > 0.f)) acc[8 * i + 2 * k] = 0.f;
                if (!(f.y > 0.f)) acc[8 * i + 2 * k + 1] = 0.f;
              }
            }
          }
          store_bf16_row<NP>(a.out + vox * NP, acc);
        }
      } else {
        if (valid) {
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

void tc_pick_tile(Dims d, bool pool, int* bx, int* by) {
  *bx = 16;
  *by = 8;
  if (pool) return;
  const long t16 = (long)((d.nx + 13) / 14) * ((d.ny + 7) / 8);
  const long t32 = (long)((d.nx + 29) / 30) * ((d.ny + 3) / 4);
  if (t32 < t16) {
    *bx = 32;
    *by = 4;
  }
}

static vie_status encode(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                         const cuuint64_t* strides, const cuuint32_t* box, CUtensorMapSwizzle swz) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return VIE_ERR_CUDA;
  }
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
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
  return encode(map, base, 4, dims, strides, box, C == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

vie_status tc_encode_planar(CUtensorMap* map, const __nv_bfloat16* base, int rows, Dims d, int nxp,
                            size_t row_stride) {
  if (nxp % 64 || rows > 256 || row_stride < (size_t)nxp * d.ny * d.nz || row_stride % 8) {
    set_error("planar tensor map: row length %d must be a multiple of 64, rows %d at most 256, row stride %zu",
              nxp, rows, row_stride);
    return VIE_ERR_INVALID;
  }
  const cuuint64_t dims[4] = {(cuuint64_t)nxp, (cuuint64_t)d.ny, (cuuint64_t)d.nz, (cuuint64_t)rows};
  const cuuint64_t strides[3] = {(cuuint64_t)nxp * 2, (cuuint64_t)nxp * 2 * d.ny, (cuuint64_t)row_stride * 2};
  const cuuint32_t box[4] = {64, 1, 1, (cuuint32_t)rows};
  return encode(map, base, 4, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

vie_status tc_encode_w(CUtensorMap* map, const __nv_bfloat16* w, int C, int N) {
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)N, 27};
  const cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * N};
  const cuuint32_t box[3] = {(cuuint32_t)C, (cuuint32_t)N, 1};
  return encode(map, w, 3, dims, strides, box, C == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
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

constexpr size_t kTcBarrierBytes = 48 * sizeof(uint64_t);

// Stages and resident CTAs per SM for a tile: the configuration with the
// most bytes of TMA loads in flight per SM, either two CTAs (each with its
// own copy of the weights) or one CTA with a deeper ring; at least three
// stages (one tile) per CTA.  (Measured on the 600 x 23 x 11 guide, warm and
// back to back: one CTA with a 14-16 stage ring beats two CTAs with 4-5.)
static void plan_stages(size_t fixed, size_t stage, const DevInfo& d, int* stages, int* per_sm) {
  const size_t sm = (size_t)d.smem_sm, rsv = (size_t)d.smem_reserved;
  *stages = 0;
  *per_sm = 0;
  size_t best = 0;
  for (int ctas = 1; ctas <= 2; ++ctas)
    for (int s = kTcMaxStages; s >= 3; --s)
      if (ctas * (fixed + s * stage + rsv) <= sm) {
        const size_t inflight = (size_t)ctas * s * stage;
        if (inflight >= best) {
          best = inflight;
          *stages = s;
          *per_sm = ctas;
        }
        break;
      }
}

template <int C, int NP, int MODE>
static vie_status launch_conv(const CUtensorMap& A, const CUtensorMap& W, TcConvArgs args, cudaStream_t s) {
  static bool configured = false;
  auto kern = conv_tc_kernel<C, NP, MODE>;
  const DevInfo& dv = dev_info();
  const size_t fixed = 1024 + 27 * (size_t)NP * C * 2 + kTcBarrierBytes;
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
  const int bxo = args.bx - 2;
  const long ntiles = (long)((d.nx + bxo - 1) / bxo) * ((d.ny + args.by - 1) / args.by) * d.nz;
  long grid = (long)dv.sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return VIE_OK;
  VIE_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(kTcThreads), smem, s, A, W, args));
  return VIE_OK;
}

vie_status tc_conv(const CUtensorMap& A, const CUtensorMap& W, int C, int NP, int mode, const TcConvArgs& args,
                   cudaStream_t s) {
  if (!((args.bx == 16 && args.by == 8) || (args.bx == 32 && args.by == 4)) ||
      (mode == TC_RELU_POOL && args.bx != 16)) {
    set_error("tensor-core convolution: unsupported tile %d x %d for mode %d", args.bx, args.by, mode);
    return VIE_ERR_INVALID;
  }
  if (C == 16 && NP == 32 && mode == TC_RELU_POOL) return launch_conv<16, 32, TC_RELU_POOL>(A, W, args, s);
  if (C == 32 && NP == 32 && mode == TC_RELU_POOL) return launch_conv<32, 32, TC_RELU_POOL>(A, W, args, s);
  if (C == 32 && NP == 32 && mode == TC_RELU_UPADD) return launch_conv<32, 32, TC_RELU_UPADD>(A, W, args, s);
  if (C == 32 && NP == 32 && mode == TC_RELU_BF16) return launch_conv<32, 32, TC_RELU_BF16>(A, W, args, s);
  if (C == 32 && NP == 16 && mode == TC_UNPACK_C64) return launch_conv<32, 16, TC_UNPACK_C64>(A, W, args, s);
  if (C == 32 && NP == 16 && mode == TC_UNPACK_C128) return launch_conv<32, 16, TC_UNPACK_C128>(A, W, args, s);
  if (C == 32 && NP == 16 && mode == TC_LINEAR_F32) return launch_conv<32, 16, TC_LINEAR_F32>(A, W, args, s);
  if (C == 16 && NP == 32 && mode == TC_GRAD_BF16) return launch_conv<16, 32, TC_GRAD_BF16>(A, W, args, s);
  if (C == 32 && NP == 32 && mode == TC_GRAD_BF16) return launch_conv<32, 32, TC_GRAD_BF16>(A, W, args, s);
  set_error("no tensor-core convolution for C=%d NP=%d mode=%d", C, NP, mode);
  return VIE_ERR_INVALID;
}

// ---------------------------------------------------------------------------
// channels-last BF16 element-wise steps
// ---------------------------------------------------------------------------
static unsigned grid_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

// sum |v|^2 over the 3 V entries as kTcNormBlocks partial sums (no atomics);
// four independent loads in flight per thread
template <typename V>
__global__ void __launch_bounds__(256) sumsq_partial_kernel(const V* __restrict__ v, size_t n,
                                                            double* __restrict__ part) {
  pdl_launch_dependents();
  pdl_wait();
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    V a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = v[i + k * stride];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc += (double)a[k].x * a[k].x + (double)a[k].y * a[k].y;
  }
  for (; i < n; i += stride) {
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
  // total of the partial sums: one load per thread, then a block reduction
  __shared__ double red[8];
  __shared__ double tot;
  double t = 0.0;
  for (int i = threadIdx.x; i < kTcNormBlocks; i += blockDim.x) t += part[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
    tot = u;
    if (blockIdx.x == 0) part[kTcNormBlocks] = u;
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

template <typename V>
vie_status tc_pack_input(const V* v, const double2* chi, Dims d, double* part, __nv_bfloat16* X, cudaStream_t s) {
  VIE_CUDA_TRY(launch_pdl(sumsq_partial_kernel<V>, dim3(kTcNormBlocks), dim3(256), 0, s, v, 3 * d.vox(), part));
  VIE_CUDA_TRY(launch_pdl(pack_cl_kernel<V>, dim3(grid_for(d.vox())), dim3(256), 0, s, v, chi, d.vox(), part, X));
  return VIE_OK;
}
template vie_status tc_pack_input<float2>(const float2*, const double2*, Dims, double*, __nv_bfloat16*, cudaStream_t);
template vie_status tc_pack_input<double2>(const double2*, const double2*, Dims, double*, __nv_bfloat16*,
                                           cudaStream_t);

}  // namespace vie
