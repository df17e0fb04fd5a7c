// Internal interface of the U-Net post-corrector's kernels (unet_conv.cu, unet.cu).
#pragma once

#include <stdint.h>

namespace fr3d {

constexpr float kLeaky = 0.01f;   // slope of leaky ReLU for negative inputs

enum ConvMode { kConvFwd = 0, kConvDgradMask = 1, kConvDgradPlain = 2 };

// One 3 x 3 x 3 convolution (or its input gradient) over CP tensors (see unet_conv.cu).  Tensors are
// byte pointers to [B][chunks][Vs][8] BF16; x_off / y_off / mask_off select a channel-chunk range of a
// larger tensor (the concatenations of the decoder).
struct ConvArgs {
  const unsigned char* x;
  int x_chunks, x_off, Cin;
  const unsigned char* wimg;   // [9 (a, e)][Cin / 16][3 (f)][N][2 chunks][8][8] BF16, K-major core matrices
  int N;
  unsigned char* y;
  int y_chunks, y_off;
  const float* bias;           // kConvFwd: [N] (may be null)
  const unsigned char* mask;   // kConvDgradMask: the tensor whose leaky derivative multiplies the result
  int mask_chunks, mask_off;
  int mode;
  int B, D, H, W, Hp, Wp;
  long Vs, p_first, p_last;
  int ntiles;                  // 128-position tiles per sample covering [p_first, p_last]
  int* err;                    // FR3D_INFO_TIMEOUT on a bounded wait that gave up (may be null)
};

// Weight gradient partials: for every voxel range r, tap and (o, c): sum over the range of G[p][o] X[p + s][c].
struct WgradArgs {
  const unsigned char* g;      // output gradient (pre-activation), Cout channels
  int g_chunks, g_off, Cout;
  const unsigned char* x;      // layer input, Cin channels
  int x_chunks, x_off, Cin;
  int ndw;                     // 3: the three f taps stacked in the rows (3 Cout <= 128); 1: one tap per CTA
  int B, Hp, Wp;
  long Vs, p_first, p_last, range;
  int ranges_per_sample;
  float* partials;             // [B * ranges_per_sample][27][Cout][Cin]
  int* err;
};

int conv3_launch(const ConvArgs& a, cudaStream_t st);
int wgrad3_launch(const WgradArgs& a, cudaStream_t st);
int wgrad_ranges_per_sample(long p_first, long p_last, long range);

}  // namespace fr3d
