// tsf_grid.cu -- launcher of the whole-GPU (cooperative) kernels.
#include <algorithm>
#include <mutex>

#include "tsf_grid.cuh"
#include "tsf_kernels.cuh"

namespace tsf {

namespace {
std::mutex g_coop;
}

cudaError_t cooperative_launch(const void* fn, dim3 grid, dim3 block, void** args, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_coop);
  cudaError_t e = cudaLaunchCooperativeKernel(fn, grid, block, args, 0, st);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaStreamSynchronize(st);
}

int cooperative_blocks(const void* fn, int threads) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0);
  return per > 0 ? std::min(sms, 128) : 0;
}

}  // namespace tsf
