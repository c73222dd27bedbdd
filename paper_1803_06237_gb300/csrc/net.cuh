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

// The network's layers and the parameter layout (FP32 master copy, BF16
// copy at the same offsets): per layer w[co][ci][27] then b[co].
constexpr int kNumLayers = 8;
struct LayerDef { int ci, co; };
// enc0..enc3, dec2, dec1, dec0, out
constexpr LayerDef kLayerDefs[kNumLayers] = {{8, 32}, {32, 32}, {32, 32}, {32, 32},
                                             {32, 32}, {32, 32}, {32, 32}, {32, 6}};
enum { ENC0 = 0, ENC1, ENC2, ENC3, DEC2, DEC1, DEC0, OUTL };
// level (pooling depth) of each layer
constexpr int kLayerLevel[kNumLayers] = {0, 1, 2, 3, 2, 1, 0, 0};

inline size_t layer_w_off(int l) {
  size_t off = 0;
  for (int i = 0; i < l; ++i) off += (size_t)kLayerDefs[i].co * kLayerDefs[i].ci * 27 + kLayerDefs[i].co;
  return off;
}
inline size_t layer_b_off(int l) { return layer_w_off(l) + (size_t)kLayerDefs[l].co * kLayerDefs[l].ci * 27; }
inline size_t total_params() { return layer_w_off(kNumLayers); }

// tensor-core weight layout wp[tap][N][C] of each layer (forward) and of its
// flipped transpose (backward data: N = the layer's inputs, C = its outputs)
inline size_t pack_size(int l) { return (size_t)27 * tc_npad(kLayerDefs[l].co) * tc_cpad(kLayerDefs[l].ci); }
inline size_t pack_off(int l) {
  size_t off = 0;
  for (int i = 0; i < l; ++i) off += pack_size(i);
  return off;
}
inline size_t packf_size(int l) { return (size_t)27 * tc_npad(kLayerDefs[l].ci) * tc_cpad(kLayerDefs[l].co); }
inline size_t packf_off(int l) {
  size_t off = 0;
  for (int i = 0; i < l; ++i) off += packf_size(i);
  return off;
}

// Epilogues of the tensor-core convolution.
enum TcMode {
  TC_RELU_BF16 = 0,   // out[vox][32] = bf16(relu(acc + bias))
  TC_UNPACK_C64 = 1,  // z_c = v_c + (y_c + i y_{3+c}) / s, complex64 planar
  TC_UNPACK_C128 = 2, // the same in complex128
  TC_RELU_POOL = 3,   // as TC_RELU_BF16, and out2 = the 2 x 2 (y, x) average of out (coarse level d2)
  TC_RELU_UPADD = 4,  // out2[fine] = bf16(bf16(relu(acc + bias)) + skip[fine]) on the 2 x 2 fine voxels
                      // of each voxel (fine level d2); out (if set) = bf16(relu(acc + bias))
  TC_LINEAR_F32 = 5,  // outf[vox][NP] = acc + bias in FP32 (the network output during training)
  TC_GRAD_BF16 = 6    // out[vox][NP] = bf16(acc), times (skip[vox][o] > 0) when skip is set: the input
                      // gradient of a layer (flipped weights, no bias), masked by the ReLU of its input
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
  float* outf;                  // TC_LINEAR_F32: channels-last FP32 output, NP channels
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
// Planar BF16 tensor [rows][nz][ny][nxp] (nxp a multiple of 64, rows
// row_stride elements apart, row_stride >= nz ny nxp) with the box
// {64, 1, 1, rows} and the 128-byte swizzle: one K-major operand tile of
// `rows` rows by 64 positions along x (the weight-gradient GEMM).
vie_status tc_encode_planar(CUtensorMap* map, const __nv_bfloat16* base, int rows, Dims d, int nxp,
                            size_t row_stride);

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

// Tensor-core training (train_tc.cu).  The network's buffers it uses: the
// packed forward weights, the packed flipped weights (backward data), the
// FP32 master parameters (biases), the gradient accumulators and the status
// flag.
struct TcTrainParams {
  const __nv_bfloat16* wpack;
  const __nv_bfloat16* wpackf;
  const float* master;
  float* grad;
  int* bad;
};
struct TcTrain;
// One training sample (r, e) on the grid n (nx, ny, nz) with contrast chi:
// forward, loss, backward; gradients added to P.grad, *loss (if not null)
// the sample's loss (synchronises s).
vie_status tc_train_accumulate(TcTrain** state, const TcTrainParams& P, const int n[3], const double2* chi,
                               const float2* r, const float2* e, double* loss, cudaStream_t s);
void tc_train_free(TcTrain* state);

}  // namespace vie
