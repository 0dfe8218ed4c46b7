// Kernels of the learned preconditioner: 3x3x3 convolutions as implicit
// GEMMs on the tensor cores (BF16 operands, FP32 accumulation), their
// backward passes, pooling, upsampling, loss and Adam.
//
// Layout: activations are channels-last [z][y][x][c] with c a multiple of
// 16 (BF16 for activations, FP32 for gradients); weights are
// [tap][c_out][c_in] with tap = 9 dz + 3 dy + dx, zero "same" padding.
#pragma once
#include "internal.cuh"

namespace to3d {
namespace cnn {

using bf16 = __nv_bfloat16;

struct ConvArgs {
    int Z, Y, X;
    long long nvox;
    int C1, C2;            // channels taken from in1 and in2 (concatenation), multiples of 16
    int Cout;              // multiple of 8
    const void* in1;
    const void* in2;
    const bf16* mask1;     // optional: A = in1 only where mask1 > 0 (ReLU of the forward layer)
    const bf16* W;         // [27][Cout][C1 + C2]
    const float* bias;     // [Cout] or null
    float* out_f;          // FP32 output (one of out_f / out_b)
    bf16* out_b;
    int out_cstride, out_coff;
    int accumulate, relu;
};

struct WgradArgs {
    int Z, Y, X;
    long long nvox;
    int Cout, Cin;         // multiples of 16 (Cout of the forward layer may be 8: padded 16 here)
    const float* gy;       // [v][gy_cstride] upstream gradient of the forward output
    int gy_cstride;
    const bf16* mask;      // forward output activations (ReLU mask) or null
    const void* x1;        // forward input channels [0, C1)
    const void* x2;        // forward input channels [C1, Cin)
    int C1;
    float* gw;             // [27][Cout_fwd][Cin] accumulated
    int Cout_fwd;          // actual forward C_out (rows of gw)
    float* gb;             // [Cout_fwd] accumulated, may be null
};

void conv_forward(const ConvArgs& a, bool in_fp32, cudaStream_t s);
void conv_wgrad(const WgradArgs& a, bool x_fp32, cudaStream_t s);
void transpose_flip(const bf16* W, bf16* Wt, int Cout, int Cin, cudaStream_t s);
void pool2_forward(const bf16* in, bf16* out, int Z, int Y, int X, int C, cudaStream_t s);
void pool2_backward(const float* gout, int gcs, int gco, float* gin, int Z, int Y, int X, int C,
                    int accumulate, cudaStream_t s);
void up2_forward(const bf16* in, bf16* out, int Z, int Y, int X, int C, cudaStream_t s);
void up2_backward(const float* gout, int gcs, int gco, float* gin, int Z, int Y, int X, int C,
                  int accumulate, cudaStream_t s);
void add_channels(const float* src, int scs, int sco, float* dst, long long nvox, int C,
                  int accumulate, cudaStream_t s);
void adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
          float eps, int t, cudaStream_t s);
void to_bf16(const float* src, bf16* dst, long long n, cudaStream_t s);

}  // namespace cnn
}  // namespace to3d
