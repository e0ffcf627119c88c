// learn.cuh -- the learned convergence accelerator around the pseudo-time iteration (the paper's
// convergence loop of Sec. 2.3 has no learned part; this is the project's addition): a 3-layer
// 3D convolutional network, channels 10 -> 32 -> 32 -> 5, 3x3x3 taps, SiLU between layers, zero
// padding in x and y and periodic in z.  It reads the state and the scaled residual of a block
// and predicts the state change over K = 20 pseudo-time steps.
//
// Storage: activations channels-last, bfloat16, channel counts padded to 16 or 32; weights in
// bfloat16 in the GEMM layout [tap][out][in]; FP32 accumulation on the tensor cores; FP32
// master weights and Adam moments.  Host parameter layout (FP32, 40677 values): per layer
// W[out][in][tap] then b[out], tap t = 9 (dz+1) + 3 (dy+1) + (dx+1).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gbcfd {
namespace learn {

constexpr int K_STEPS = 20;
constexpr int NTAP = 27;
constexpr int C0 = 10, C1 = 32, C2 = 32, C3 = 5;   // channels
constexpr int P0 = 16, P1 = 32, P2 = 32, P3 = 8;   // padded channel counts of the stored tensors
constexpr int NW1 = C1 * C0 * NTAP, NW2 = C2 * C1 * NTAP, NW3 = C3 * C2 * NTAP;
constexpr int OFF_W1 = 0, OFF_B1 = NW1, OFF_W2 = NW1 + C1, OFF_B2 = OFF_W2 + NW2, OFF_W3 = OFF_B2 + C2,
              OFF_B3 = OFF_W3 + NW3, NPARAM = OFF_B3 + C3;  // 40677
constexpr float STATE_GAIN = 10.0f;
constexpr int TILE_X = 32, TILE_Y = 4;               // 128 cells per weight-gradient tile
constexpr int BOX_X = TILE_X + 2, BOX_Y = TILE_Y + 2, BOX_Z = 3;
constexpr int BOX = BOX_X * BOX_Y * BOX_Z;           // input cells a tile reads
constexpr int NTHREADS = 256;

enum ConvMode { FWD_SILU = 0, FWD_LINEAR = 1, BWD_DSILU = 2 };

// one convolution launch over a volume of B batches of X x Y x Z cells (channels-last tensors)
struct ConvArgs {
  const __nv_bfloat16* in;   // [cell][CIP]
  const __nv_bfloat16* w;    // [27][N][CIP] (N = the MMA width: COP, or 16 for the 8-channel output)
  const float* bias;         // [COP] (forward modes)
  void* out;                 // bf16 [cell][COP] (FWD_SILU, BWD_DSILU) or f32 [cell][COP] (FWD_LINEAR)
  float* zsave;              // FWD_SILU: pre-activation f32 [cell][COP] when not null (training)
  const float* zprev;        // BWD_DSILU: the pre-activation whose SiLU derivative multiplies
  int X, Y, Z, B, zper;
};

// the accelerator's device arrays (carved from one caller buffer)
struct Net {
  float *w, *m, *v, *grad;            // master parameters, Adam moments, gradient (NPARAM each)
  __nv_bfloat16 *w1, *w2, *w3;        // forward GEMM layouts [27][N][CIP] (w3: N = 16, 5 used)
  __nv_bfloat16 *w3b, *w2b;           // backward-data layouts (taps mirrored, in/out swapped)
  float *b1, *b2, *b3;                // padded biases
  float* wpart;                       // weight-gradient partials [grid][NPARAM]
  int wgrid;
  int* flag;                          // FLAG_TIMEOUT when a bounded wait of a convolution gave up
};

cudaError_t launch_conv(int layer, int mode, const ConvArgs& a, int* flag, cudaStream_t s);
cudaError_t launch_wgrad(int layer, const __nv_bfloat16* a, const __nv_bfloat16* g, const Net& n, int X, int Y,
                         int Z, int B, int zper, cudaStream_t s);
cudaError_t launch_grad_reduce(const Net& n, cudaStream_t s);
cudaError_t launch_adam(const Net& n, float lr, int step, cudaStream_t s);
cudaError_t launch_pack(const Net& n, cudaStream_t s);
cudaError_t launch_loss(const float* y, const float* t, __nv_bfloat16* dy, double* partial, long long cells,
                        int grid, cudaStream_t s);
cudaError_t launch_sum(const double* partial, int n, int stride, double* out, cudaStream_t s);

// block-facing kernels: features from a block's padded state Q (f64), compact residual R (f64)
// and local time steps; the saved compact state; prediction and target
struct BlockView {
  int nx, ny, nz;
  long long field, fieldf;   // padded field sizes (f64 / f32 elements)
  int px, pxf;
  double* q;                 // padded f64 state Q^n
  float* sh;                 // mixed path: padded f32 shadow of Q^n (or null)
  const void* dtl;           // local time steps (f64 or f32 padded field), or null: use *dt
  int dtl_f32;
  const double* dt;          // the global step (device) when dtl is null
  double qinf[5], ref[5];    // free stream (conserved) and reference scales
};
cudaError_t launch_feature_stats(const BlockView& v, const double* R, double* partial, int grid, cudaStream_t s);
cudaError_t launch_features(const BlockView& v, const double* R, const double* stats, __nv_bfloat16* x,
                            double* qsave, cudaStream_t s);
cudaError_t launch_apply(const BlockView& v, const float* y, const double* qsave, const double* stats, int revert,
                         cudaStream_t s, double alpha = 1.0);
cudaError_t launch_target(const BlockView& v, const double* qsave, const double* stats, float* t, cudaStream_t s);

}  // namespace learn
}  // namespace gbcfd
