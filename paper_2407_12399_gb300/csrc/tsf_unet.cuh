// tsf_unet.cuh -- declarations shared by the warm-start network's kernels
// (k_unet.cu) and its C ABI (tsf_unet.cu).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace tsf {
namespace unet {

constexpr int kConvStages = 4;                 // TMA/MMA pipeline depth of the convolution
constexpr size_t kConvMaxSmem = 200 * 1024;    // dynamic shared memory limit set for it
constexpr uint32_t kUnetErrSpin = 1u << 5;     // a bounded wait gave up (same bit as the solver's)

enum ConvMode { kConvForward = 0, kConvDgrad = 1 };

// One 3x3x3 'same' convolution as an implicit GEMM (k_conv_tc).  The caller
// fills the first group; launch_conv derives the rest.
struct ConvArgs {
  int lx, ly, lz;     // grid of input and output (the output of an `up` launch is 2x)
  int cout;           // output channels (multiple of 16, <= 128)
  int mode;           // kConvForward: relu(acc + bias); kConvDgrad: acc masked by mask > 0
  int up;             // forward only: store every voxel to its 2x2x2 block of a 2x grid
  void* out;          // output planes (bf16)
  int64_t out_plane0; // first output plane
  const void* mask;   // dgrad: activation whose ReLU masks the output (may be null)
  int64_t mask_plane0;
  const float* bias;  // forward: cout biases (bf16 values)
  const __nv_bfloat16* wpack;  // stage-packed weights (k_pack_weights)
  uint32_t* status;   // device status word (kUnetErrSpin)
  // derived
  int chunks, taps_per_stage, kchunks, nstages, tmem_cols, bx, by;
};

int launch_conv(const ConvArgs& a, const void* in_planes, int in_chunks, cudaStream_t st);
size_t conv_smem_bytes(int kchunks, int cout);
void tile_shape(int lx, int& bx, int& by);

void launch_pack_input(const float* f, float tau, int64_t nv, void* x, cudaStream_t st);
void launch_avgpool(const void* in, int in_plane0, int planes, int lx, int ly, int lz, void* out, cudaStream_t st);
void launch_upsample_back(const void* g, int g_plane0, int planes, int lx, int ly, int lz, const void* act_up,
                          int act_plane0, void* out, cudaStream_t st);
void launch_skip_back(const void* gs, int gs_plane0, const void* gp, const void* s, int s_plane0, int planes, int lx,
                      int ly, int lz, void* out, cudaStream_t st);
void launch_head_forward(const void* u1, const float* hw, int64_t nv, const float* f, float* g0, cudaStream_t st);
int head_blocks(int64_t nv);
void launch_head_backward(const void* u1, const float* hw, int64_t nv, const float* f, const float* g, void* gz,
                          double* partial, double* loss, float* grad, int64_t hw_off, int64_t hb_off, cudaStream_t st);
int64_t wgrad_partial_floats(int64_t nv, int cout, int cin);
int64_t bias_partial_floats(int64_t nv, int cout);
void launch_wgrad(const void* x, int x_plane0, int cin, int cin_real, const void* gz, int cout, int lx, int ly, int lz,
                  float* partial, float* gw, float* bpartial, float* gb, cudaStream_t st);
void launch_pack_weights(const float* w, int cout_f, int cin_real, int cin_pad, int transpose, void* pack,
                         cudaStream_t st);
int64_t pack_elems(int cout_f, int cin_pad, int transpose);
void launch_round_bf16(const float* in, int64_t n, float* out, cudaStream_t st);
void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                 float eps, float bc1, float bc2, cudaStream_t st);
void launch_unpack_planes(const void* in, int plane0, int c_real, int64_t nv, float* out, cudaStream_t st);

}  // namespace unet
}  // namespace tsf
