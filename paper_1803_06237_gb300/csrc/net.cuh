// Shared declarations of the learned preconditioner's kernels: the FP32
// training path in precond.cu and the tensor-core inference path in
// conv_tc.cu.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "vie_internal.cuh"

namespace vie {

struct Dims {
  int nz, ny, nx;
  __host__ __device__ size_t vox() const { return (size_t)nz * ny * nx; }
};

// Padded channel counts of the tensor-core convolution: the input channels
// (the K extent of one tap) are 16 or 32, the output channels (N) 16 or 32.
inline int tc_cpad(int ci) { return ci <= 16 ? 16 : 32; }
inline int tc_npad(int co) { return co <= 16 ? 16 : 32; }

// Epilogues of the tensor-core convolution.
enum TcMode {
  TC_RELU_BF16 = 0,   // out[vox][32] = bf16(relu(acc + bias))
  TC_UNPACK_C64 = 1,  // z_c = v_c + (y_c + i y_{3+c}) / s, complex64 planar
  TC_UNPACK_C128 = 2, // the same in complex128
  TC_RELU_POOL = 3,   // as TC_RELU_BF16, and out2 = the 2 x 2 (y, x) average of out (coarse level d2)
  TC_RELU_UPADD = 4   // out2[fine] = bf16(bf16(relu(acc + bias)) + skip[fine]) on the 2 x 2 fine voxels
                      // of each voxel (fine level d2); out itself is not written
};

struct TcConvArgs {
  Dims d;                       // grid of this level
  Dims d2;                      // grid of out2 (coarse for TC_RELU_POOL, fine for TC_RELU_UPADD)
  int bx, by;                   // tile: bx input x columns (bx - 2 outputs) times by rows in y (bx * by = 128)
  int stages;                   // depth of the TMA ring (set by tc_conv)
  const float* bias;            // co biases (FP32)
  int co;                       // real output channels
  __nv_bfloat16* out;           // channels-last output, 32 channels
  __nv_bfloat16* out2;          // pooled / upsampled-and-added output, 32 channels
  const __nv_bfloat16* skip;    // TC_RELU_UPADD: the fine-level skip tensor
  const void* v;                // TC_UNPACK_*: the preconditioned vector (3 planar components)
  void* z;                      //              and the result
  const double* sumsq;          //              sum |v|^2 (the input scale)
  int* bad;                     // non-finite output (1) or a wait that timed out (2)
};

// Tile for a level: bx = 16 or 32 input columns (a one-voxel halo on each
// side, bx - 2 outputs) and by = 128 / bx rows; the fewest tiles wins.
// Pooling epilogues need bx = 16 (a 2 x 2 block inside one warp).
void tc_pick_tile(Dims d, bool pool, int* bx, int* by);

// Tensor maps: channels-last BF16 activation [nz][ny][nx][C] with the box
// {C, bx, by + 2, 1}; packed weights [27][N][C] with the box {C, N, 1}.
vie_status tc_encode_act(CUtensorMap* map, const __nv_bfloat16* base, int C, Dims d, int bx, int by);
vie_status tc_encode_w(CUtensorMap* map, const __nv_bfloat16* w, int C, int N);

// One 3x3x3 convolution (zero padding) as an implicit GEMM on the tensor
// cores: M = the 128 input positions of a tile, N = 3 x the output channels
// (one block per dx tap), K = 9 (dz, dy) taps x C; the epilogue adds the dx
// blocks of neighbouring positions.
vie_status tc_conv(const CUtensorMap& A, const CUtensorMap& W, int C, int N, int mode, const TcConvArgs& args,
                   cudaStream_t s);

// Channels-last BF16 helpers of the inference path.  tc_pack_input sums
// |v|^2 into kTcNormBlocks partials (part[0 .. kTcNormBlocks), total in
// part[kTcNormBlocks]) and packs the scaled input X[vox][16].
constexpr int kTcNormBlocks = 256;
template <typename V>
vie_status tc_pack_input(const V* v, const double2* chi, Dims d, double* part, __nv_bfloat16* X, cudaStream_t s);

}  // namespace vie
