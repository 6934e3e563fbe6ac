// tsf_unet.cu -- C ABI of the learned warm start (include/tsf.h,
// tsf_unet_*): the network's parameters and buffers, and the order of its
// layers.  Every computation runs in the kernels of k_unet.cu.
//
// Network (the paper has no learned component; these are this library's
// choices): a 3-level 3D U-Net on an (lz, ly, lx) grid with each side a
// multiple of 4, channels 16/32/64, per level two 3x3x3 'same' convolutions
// with bias and ReLU, 2x2x2 average pooling down, nearest x2 upsampling up,
// the skip features concatenated after the upsampled ones, a 1x1 head; input
// channels f and the constant threshold tau; output g0 = f + head.
// Parameters are kept in fp32 (the Adam master copy) and used in bf16.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/tsf.h"
#include "tsf_kernels.cuh"
#include "tsf_unet.cuh"

using namespace tsf::unet;

namespace {

struct Layer {
  int cout, cin_real, cin_pad;
  int64_t w_off, b_off;
};

enum { E1A, E1B, E2A, E2B, E3A, E3B, D2A, D2B, D1A, D1B, NCONV };

struct Net {
  Layer L[NCONV];
  int64_t head_w, head_b, nparams;
  Net() {
    const int spec[NCONV][3] = {{16, 2, 8},   {16, 16, 16}, {32, 16, 16}, {32, 32, 32}, {64, 32, 32},
                                {64, 64, 64}, {32, 96, 96}, {32, 32, 32}, {16, 48, 48}, {16, 16, 16}};
    int64_t off = 0;
    for (int i = 0; i < NCONV; ++i) {
      L[i] = {spec[i][0], spec[i][1], spec[i][2], off, off + (int64_t)spec[i][0] * spec[i][1] * 27};
      off = L[i].b_off + spec[i][0];
    }
    head_w = off;
    head_b = off + 16;
    nparams = off + 17;
  }
};
const Net kNet;

template <class T>
cudaError_t dalloc(T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)n);
}
template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

}  // namespace

struct tsf_unet {
  int device = 0;
  cudaStream_t st = nullptr;
  uint32_t* status = nullptr;
  float *params = nullptr, *rounded = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* pack_f[NCONV] = {};
  __nv_bfloat16* pack_d[NCONV] = {};
  int64_t adam_t = 0;
  // buffers for the current grid
  int lx = 0, ly = 0, lz = 0;
  uint4 *xin = nullptr, *a1a = nullptr, *cat1 = nullptr, *p1 = nullptr, *a2a = nullptr, *cat2 = nullptr, *p2 = nullptr,
        *a3a = nullptr, *a3b = nullptr, *a2d = nullptr, *a2b = nullptr, *a1d = nullptr, *u1 = nullptr;
  uint4 *gzA1 = nullptr, *gzB1 = nullptr, *gcat1 = nullptr, *gzA2 = nullptr, *gzB2 = nullptr, *gcat2 = nullptr,
        *gzA3 = nullptr, *gzB3 = nullptr, *gp2 = nullptr, *gp1 = nullptr;
  float *fbuf = nullptr, *gbuf = nullptr, *g0 = nullptr, *wpart = nullptr, *bpart = nullptr;
  double *hpart = nullptr, *loss = nullptr;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void free_grid(tsf_unet* U) {
  uint4** bufs[] = {&U->xin, &U->a1a, &U->cat1, &U->p1, &U->a2a, &U->cat2, &U->p2, &U->a3a, &U->a3b, &U->a2d,
                    &U->a2b, &U->a1d, &U->u1, &U->gzA1, &U->gzB1, &U->gcat1, &U->gzA2, &U->gzB2, &U->gcat2,
                    &U->gzA3, &U->gzB3, &U->gp2, &U->gp1};
  for (auto b : bufs) dfree(*b);
  dfree(U->fbuf);
  dfree(U->gbuf);
  dfree(U->g0);
  dfree(U->wpart);
  dfree(U->bpart);
  dfree(U->hpart);
  U->lx = U->ly = U->lz = 0;
}

// Buffers for a grid; `train` adds the backward buffers.
int ensure_grid(tsf_unet* U, int lx, int ly, int lz, bool train) {
  if (lx < 8 || ly < 8 || lz < 8 || lx % 4 || ly % 4 || lz % 4) return TSF_EINVAL;
  const bool have_train = U->gzA1 != nullptr;
  if (U->lx == lx && U->ly == ly && U->lz == lz && (!train || have_train)) return TSF_OK;
  free_grid(U);
  const int64_t n1 = (int64_t)lx * ly * lz, n2 = n1 / 8, n3 = n2 / 8;
  cudaError_t e = cudaSuccess;
  auto A = [&](uint4** p, int64_t n) {
    if (e == cudaSuccess) e = dalloc(p, n);
  };
  A(&U->xin, n1);
  A(&U->a1a, 2 * n1);
  A(&U->cat1, 6 * n1);
  A(&U->p1, 2 * n2);
  A(&U->a2a, 4 * n2);
  A(&U->cat2, 12 * n2);
  A(&U->p2, 4 * n3);
  A(&U->a3a, 8 * n3);
  A(&U->a3b, 8 * n3);
  A(&U->a2d, 4 * n2);
  A(&U->a2b, 4 * n2);
  A(&U->a1d, 2 * n1);
  A(&U->u1, 2 * n1);
  if (e == cudaSuccess) e = dalloc(&U->fbuf, n1);
  if (e == cudaSuccess) e = dalloc(&U->g0, n1);
  if (train) {
    A(&U->gzA1, 2 * n1);
    A(&U->gzB1, 2 * n1);
    A(&U->gcat1, 6 * n1);
    A(&U->gzA2, 4 * n2);
    A(&U->gzB2, 4 * n2);
    A(&U->gcat2, 12 * n2);
    A(&U->gzA3, 8 * n3);
    A(&U->gzB3, 8 * n3);
    A(&U->gp2, 4 * n3);
    A(&U->gp1, 2 * n2);
    if (e == cudaSuccess) e = dalloc(&U->gbuf, n1);
    int64_t wp = 0, bp = 0;
    const int64_t nv_of[NCONV] = {n1, n1, n2, n2, n3, n3, n2, n2, n1, n1};
    for (int i = 0; i < NCONV; ++i) {
      wp = std::max(wp, wgrad_partial_floats(nv_of[i], kNet.L[i].cout, kNet.L[i].cin_pad));
      bp = std::max(bp, bias_partial_floats(nv_of[i], kNet.L[i].cout));
    }
    if (e == cudaSuccess) e = dalloc(&U->wpart, wp);
    if (e == cudaSuccess) e = dalloc(&U->bpart, bp);
    if (e == cudaSuccess) e = dalloc(&U->hpart, (int64_t)head_blocks(n1) * 18);
  }
  if (e != cudaSuccess) {
    free_grid(U);
    cudaGetLastError();
    return TSF_ENOMEM;
  }
  U->lx = lx;
  U->ly = ly;
  U->lz = lz;
  return TSF_OK;
}

// bf16 operands from the fp32 master parameters.
void repack(tsf_unet* U) {
  for (int i = 0; i < NCONV; ++i) {
    const Layer& l = kNet.L[i];
    launch_pack_weights(U->params + l.w_off, l.cout, l.cin_real, l.cin_pad, 0, U->pack_f[i], U->st);
    if (i != E1A) launch_pack_weights(U->params + l.w_off, l.cout, l.cin_real, l.cin_pad, 1, U->pack_d[i], U->st);
  }
  launch_round_bf16(U->params, kNet.nparams, U->rounded, U->st);
}

int conv(tsf_unet* U, int layer, int mode, const uint4* in, int in_chunks, int lx, int ly, int lz, uint4* out,
         int64_t out_plane0, int up, const uint4* mask, int64_t mask_plane0) {
  const Layer& l = kNet.L[layer];
  ConvArgs a{};
  a.lx = lx;
  a.ly = ly;
  a.lz = lz;
  a.mode = mode;
  a.up = up;
  a.out = out;
  a.out_plane0 = out_plane0;
  a.mask = mask;
  a.mask_plane0 = mask_plane0;
  a.status = U->status;
  if (mode == kConvForward) {
    a.cout = l.cout;
    a.bias = U->rounded + l.b_off;
    a.wpack = U->pack_f[layer];
  } else {
    a.cout = l.cin_pad;
    a.bias = nullptr;
    a.wpack = U->pack_d[layer];
  }
  tsf::note_launch();
  return launch_conv(a, in, in_chunks, U->st) == 0 ? TSF_OK : TSF_ECUDA;
}

// Forward pass from U->fbuf; `keep` also stores e3b and d2b without
// upsampling (their separate copies are read by the debug output only).
int forward(tsf_unet* U, float tau, bool keep) {
  const int lx = U->lx, ly = U->ly, lz = U->lz;
  const int64_t n1 = (int64_t)lx * ly * lz;
  const int x2 = lx / 2, y2 = ly / 2, z2 = lz / 2, x3 = lx / 4, y3 = ly / 4, z3 = lz / 4;
  cudaStream_t st = U->st;
  int r = TSF_OK;
  launch_pack_input(U->fbuf, tau, n1, U->xin, st);
  if (!r) r = conv(U, E1A, kConvForward, U->xin, 1, lx, ly, lz, U->a1a, 0, 0, nullptr, 0);
  if (!r) r = conv(U, E1B, kConvForward, U->a1a, 2, lx, ly, lz, U->cat1, 4, 0, nullptr, 0);
  launch_avgpool(U->cat1, 4, 2, lx, ly, lz, U->p1, st);
  if (!r) r = conv(U, E2A, kConvForward, U->p1, 2, x2, y2, z2, U->a2a, 0, 0, nullptr, 0);
  if (!r) r = conv(U, E2B, kConvForward, U->a2a, 4, x2, y2, z2, U->cat2, 8, 0, nullptr, 0);
  launch_avgpool(U->cat2, 8, 4, x2, y2, z2, U->p2, st);
  if (!r) r = conv(U, E3A, kConvForward, U->p2, 4, x3, y3, z3, U->a3a, 0, 0, nullptr, 0);
  if (!r) r = conv(U, E3B, kConvForward, U->a3a, 8, x3, y3, z3, U->cat2, 0, 1, nullptr, 0);
  if (!r && keep) r = conv(U, E3B, kConvForward, U->a3a, 8, x3, y3, z3, U->a3b, 0, 0, nullptr, 0);
  if (!r) r = conv(U, D2A, kConvForward, U->cat2, 12, x2, y2, z2, U->a2d, 0, 0, nullptr, 0);
  if (!r) r = conv(U, D2B, kConvForward, U->a2d, 4, x2, y2, z2, U->cat1, 0, 1, nullptr, 0);
  if (!r && keep) r = conv(U, D2B, kConvForward, U->a2d, 4, x2, y2, z2, U->a2b, 0, 0, nullptr, 0);
  if (!r) r = conv(U, D1A, kConvForward, U->cat1, 6, lx, ly, lz, U->a1d, 0, 0, nullptr, 0);
  if (!r) r = conv(U, D1B, kConvForward, U->a1d, 2, lx, ly, lz, U->u1, 0, 0, nullptr, 0);
  return r;
}

void wgrad(tsf_unet* U, int layer, const uint4* x, int x_plane0, const uint4* gz, int lx, int ly, int lz) {
  const Layer& l = kNet.L[layer];
  launch_wgrad(x, x_plane0, l.cin_pad, l.cin_real, gz, l.cout, lx, ly, lz, U->wpart, U->grad + l.w_off, U->bpart,
               U->grad + l.b_off, U->st);
}

// Backward pass of mean((g0 - g)^2) after forward(); parameter gradients in
// U->grad (reference layout), the loss in U->loss.  `keep` (may be null)
// receives every convolution's pre-activation gradient as fp32 (C, z, y, x),
// in the order d1b d1a d2b d2a e3b e3a e2b e2a e1b e1a.
int backward(tsf_unet* U, float* keep) {
  const int lx = U->lx, ly = U->ly, lz = U->lz;
  const int64_t n1 = (int64_t)lx * ly * lz, n2 = n1 / 8, n3 = n2 / 8;
  const int x2 = lx / 2, y2 = ly / 2, z2 = lz / 2, x3 = lx / 4, y3 = ly / 4, z3 = lz / 4;
  cudaStream_t st = U->st;
  int64_t ko = 0;
  auto put = [&](const uint4* b, int c, int64_t nv) {
    if (!keep) return;
    launch_unpack_planes(b, 0, c, nv, keep + ko, st);
    ko += c * nv;
  };
  int r = TSF_OK;
  launch_head_backward(U->u1, U->rounded + kNet.head_w, n1, U->fbuf, U->gbuf, U->gzA1, U->hpart, U->loss, U->grad,
                       kNet.head_w, kNet.head_b, st);
  put(U->gzA1, 16, n1);
  wgrad(U, D1B, U->a1d, 0, U->gzA1, lx, ly, lz);
  if (!r) r = conv(U, D1B, kConvDgrad, U->gzA1, 2, lx, ly, lz, U->gzB1, 0, 0, U->a1d, 0);
  put(U->gzB1, 16, n1);
  wgrad(U, D1A, U->cat1, 0, U->gzB1, lx, ly, lz);
  if (!r) r = conv(U, D1A, kConvDgrad, U->gzB1, 2, lx, ly, lz, U->gcat1, 0, 0, nullptr, 0);
  launch_upsample_back(U->gcat1, 0, 4, lx, ly, lz, U->cat1, 0, U->gzA2, st);
  put(U->gzA2, 32, n2);
  wgrad(U, D2B, U->a2d, 0, U->gzA2, x2, y2, z2);
  if (!r) r = conv(U, D2B, kConvDgrad, U->gzA2, 4, x2, y2, z2, U->gzB2, 0, 0, U->a2d, 0);
  put(U->gzB2, 32, n2);
  wgrad(U, D2A, U->cat2, 0, U->gzB2, x2, y2, z2);
  if (!r) r = conv(U, D2A, kConvDgrad, U->gzB2, 4, x2, y2, z2, U->gcat2, 0, 0, nullptr, 0);
  launch_upsample_back(U->gcat2, 0, 8, x2, y2, z2, U->cat2, 0, U->gzA3, st);
  put(U->gzA3, 64, n3);
  wgrad(U, E3B, U->a3a, 0, U->gzA3, x3, y3, z3);
  if (!r) r = conv(U, E3B, kConvDgrad, U->gzA3, 8, x3, y3, z3, U->gzB3, 0, 0, U->a3a, 0);
  put(U->gzB3, 64, n3);
  wgrad(U, E3A, U->p2, 0, U->gzB3, x3, y3, z3);
  if (!r) r = conv(U, E3A, kConvDgrad, U->gzB3, 8, x3, y3, z3, U->gp2, 0, 0, nullptr, 0);
  launch_skip_back(U->gcat2, 8, U->gp2, U->cat2, 8, 4, x2, y2, z2, U->gzA2, st);
  put(U->gzA2, 32, n2);
  wgrad(U, E2B, U->a2a, 0, U->gzA2, x2, y2, z2);
  if (!r) r = conv(U, E2B, kConvDgrad, U->gzA2, 4, x2, y2, z2, U->gzB2, 0, 0, U->a2a, 0);
  put(U->gzB2, 32, n2);
  wgrad(U, E2A, U->p1, 0, U->gzB2, x2, y2, z2);
  if (!r) r = conv(U, E2A, kConvDgrad, U->gzB2, 4, x2, y2, z2, U->gp1, 0, 0, nullptr, 0);
  launch_skip_back(U->gcat1, 4, U->gp1, U->cat1, 4, 2, lx, ly, lz, U->gzA1, st);
  put(U->gzA1, 16, n1);
  wgrad(U, E1B, U->a1a, 0, U->gzA1, lx, ly, lz);
  if (!r) r = conv(U, E1B, kConvDgrad, U->gzA1, 2, lx, ly, lz, U->gzB1, 0, 0, U->a1a, 0);
  put(U->gzB1, 16, n1);
  wgrad(U, E1A, U->xin, 0, U->gzB1, lx, ly, lz);
  return r;
}

int finish(tsf_unet* U) {
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return TSF_ECUDA;
  }
  uint32_t s = 0;
  if (cudaMemcpyAsync(&s, U->status, 4, cudaMemcpyDeviceToHost, U->st) != cudaSuccess) return TSF_ECUDA;
  if (cudaStreamSynchronize(U->st) != cudaSuccess) return TSF_ECUDA;
  if (s) {
    cudaMemsetAsync(U->status, 0, 4, U->st);
    cudaStreamSynchronize(U->st);
    return TSF_ETIMEOUT;
  }
  return TSF_OK;
}

int load_inputs(tsf_unet* U, const float* f, const float* g, int on_device) {
  const size_t bytes = sizeof(float) * (size_t)U->lx * U->ly * U->lz;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(U->fbuf, f, bytes, k, U->st) != cudaSuccess) return TSF_ECUDA;
  if (g && cudaMemcpyAsync(U->gbuf, g, bytes, k, U->st) != cudaSuccess) return TSF_ECUDA;
  return TSF_OK;
}

}  // namespace

extern "C" {

int64_t tsf_unet_num_params(void) { return kNet.nparams; }

int tsf_unet_create(const float* params, int64_t n, void* cuda_stream, tsf_unet** out) {
  if (!out || !params || n != kNet.nparams) return TSF_EINVAL;
  *out = nullptr;
  tsf_unet* U = new tsf_unet();
  cudaGetDevice(&U->device);
  U->st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = dalloc(&U->status, 1);
  if (e == cudaSuccess) e = dalloc(&U->params, n);
  if (e == cudaSuccess) e = dalloc(&U->rounded, n);
  if (e == cudaSuccess) e = dalloc(&U->grad, n);
  if (e == cudaSuccess) e = dalloc(&U->m, n);
  if (e == cudaSuccess) e = dalloc(&U->v, n);
  if (e == cudaSuccess) e = dalloc(&U->loss, 1);
  for (int i = 0; i < NCONV && e == cudaSuccess; ++i) {
    e = dalloc(&U->pack_f[i], pack_elems(kNet.L[i].cout, kNet.L[i].cin_pad, 0));
    if (e == cudaSuccess && i != E1A) e = dalloc(&U->pack_d[i], pack_elems(kNet.L[i].cout, kNet.L[i].cin_pad, 1));
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    tsf_unet_destroy(U);
    return TSF_ENOMEM;
  }
  cudaMemsetAsync(U->status, 0, 4, U->st);
  cudaMemsetAsync(U->grad, 0, sizeof(float) * n, U->st);
  cudaMemsetAsync(U->m, 0, sizeof(float) * n, U->st);
  cudaMemsetAsync(U->v, 0, sizeof(float) * n, U->st);
  cudaMemcpyAsync(U->params, params, sizeof(float) * n, cudaMemcpyHostToDevice, U->st);
  repack(U);
  const int r = finish(U);
  if (r != TSF_OK) {
    tsf_unet_destroy(U);
    return r;
  }
  *out = U;
  return TSF_OK;
}

int tsf_unet_destroy(tsf_unet* U) {
  if (!U) return TSF_OK;
  DeviceGuard g(U->device);
  if (U->st) cudaStreamSynchronize(U->st);
  free_grid(U);
  dfree(U->status);
  dfree(U->params);
  dfree(U->rounded);
  dfree(U->grad);
  dfree(U->m);
  dfree(U->v);
  dfree(U->loss);
  for (int i = 0; i < NCONV; ++i) {
    dfree(U->pack_f[i]);
    dfree(U->pack_d[i]);
  }
  delete U;
  return TSF_OK;
}

int tsf_unet_get_params(tsf_unet* U, float* out, int64_t n) {
  if (!U || !out || n != kNet.nparams) return TSF_EINVAL;
  DeviceGuard g(U->device);
  if (cudaMemcpyAsync(out, U->params, sizeof(float) * n, cudaMemcpyDeviceToHost, U->st) != cudaSuccess)
    return TSF_ECUDA;
  return cudaStreamSynchronize(U->st) == cudaSuccess ? TSF_OK : TSF_ECUDA;
}

int tsf_unet_forward(tsf_unet* U, int lx, int ly, int lz, const float* f, float tau, float* g0, int on_device) {
  if (!U || !f || !g0 || !std::isfinite(tau)) return TSF_EINVAL;
  DeviceGuard gd(U->device);
  int r = ensure_grid(U, lx, ly, lz, false);
  if (r) return r;
  if ((r = load_inputs(U, f, nullptr, on_device))) return r;
  if ((r = forward(U, tau, false))) return r;
  const int64_t n1 = (int64_t)lx * ly * lz;
  launch_head_forward(U->u1, U->rounded + kNet.head_w, n1, U->fbuf, U->g0, U->st);
  if (cudaMemcpyAsync(g0, U->g0, sizeof(float) * (size_t)n1, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      U->st) != cudaSuccess)
    return TSF_ECUDA;
  return finish(U);
}

int tsf_unet_gradients(tsf_unet* U, int lx, int ly, int lz, const float* f, const float* g, int on_device, float tau,
                       float* grad, double* loss) {
  if (!U || !f || !g || !std::isfinite(tau)) return TSF_EINVAL;
  DeviceGuard gd(U->device);
  int r = ensure_grid(U, lx, ly, lz, true);
  if (r) return r;
  if ((r = load_inputs(U, f, g, on_device))) return r;
  if ((r = forward(U, tau, false))) return r;
  if ((r = backward(U, nullptr))) return r;
  if (grad && cudaMemcpyAsync(grad, U->grad, sizeof(float) * kNet.nparams, cudaMemcpyDeviceToHost, U->st) != cudaSuccess)
    return TSF_ECUDA;
  if (loss && cudaMemcpyAsync(loss, U->loss, sizeof(double), cudaMemcpyDeviceToHost, U->st) != cudaSuccess)
    return TSF_ECUDA;
  return finish(U);
}

int tsf_unet_train_step(tsf_unet* U, int lx, int ly, int lz, const float* f, const float* g, int on_device, float tau,
                        float lr, double* loss) {
  if (!U || !f || !g || !std::isfinite(tau) || !(lr >= 0.0f) || !std::isfinite(lr)) return TSF_EINVAL;
  DeviceGuard gd(U->device);
  int r = ensure_grid(U, lx, ly, lz, true);
  if (r) return r;
  if ((r = load_inputs(U, f, g, on_device))) return r;
  if ((r = forward(U, tau, false))) return r;
  if ((r = backward(U, nullptr))) return r;
  U->adam_t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = (float)(1.0 - std::pow(b1, (double)U->adam_t)), bc2 = (float)(1.0 - std::pow(b2, (double)U->adam_t));
  launch_adam(U->params, U->grad, U->m, U->v, kNet.nparams, lr, (float)b1, (float)b2, 1e-8f, bc1, bc2, U->st);
  repack(U);
  if (loss && cudaMemcpyAsync(loss, U->loss, sizeof(double), cudaMemcpyDeviceToHost, U->st) != cudaSuccess)
    return TSF_ECUDA;
  return finish(U);
}

// Stored activations of every layer (fp32 copies of the bf16 values, each
// (C, z, y, x) at its level) and, when g is given, every convolution's
// pre-activation gradient, for layer-by-layer verification.
int tsf_unet_debug(tsf_unet* U, int lx, int ly, int lz, const float* f, const float* g, float tau, float* acts,
                   int64_t acts_cap, float* gz, int64_t gz_cap) {
  if (!U || !f || !acts || !std::isfinite(tau)) return TSF_EINVAL;
  DeviceGuard gd(U->device);
  const bool train = g != nullptr;
  int r = ensure_grid(U, lx, ly, lz, train);
  if (r) return r;
  const int64_t n1 = (int64_t)lx * ly * lz, n2 = n1 / 8, n3 = n2 / 8;
  // x e1a e1b e2a e2b e3a e3b d2a d2b d1a d1b g0
  const int64_t need = 2 * n1 + 16 * n1 + 16 * n1 + 32 * n2 + 32 * n2 + 64 * n3 + 64 * n3 + 32 * n2 + 32 * n2 +
                       16 * n1 + 16 * n1 + n1;
  // gradients: d1b d1a d2b d2a e3b e3a e2b e2a e1b e1a
  const int64_t need_g = 16 * n1 + 16 * n1 + 32 * n2 + 32 * n2 + 64 * n3 + 64 * n3 + 32 * n2 + 32 * n2 + 16 * n1 +
                         16 * n1;
  if (acts_cap < need || (train && (!gz || gz_cap < need_g))) return TSF_ECAPACITY;
  if ((r = load_inputs(U, f, g, 0))) return r;
  if ((r = forward(U, tau, true))) return r;
  launch_head_forward(U->u1, U->rounded + kNet.head_w, n1, U->fbuf, U->g0, U->st);
  float* tmp = nullptr;
  if (dalloc(&tmp, std::max(need, train ? need_g : 0)) != cudaSuccess) return TSF_ENOMEM;
  int64_t o = 0;
  auto put = [&](const uint4* b, int plane0, int c, int64_t nv) {
    launch_unpack_planes(b, plane0, c, nv, tmp + o, U->st);
    o += c * nv;
  };
  put(U->xin, 0, 2, n1);
  put(U->a1a, 0, 16, n1);
  put(U->cat1, 4, 16, n1);
  put(U->a2a, 0, 32, n2);
  put(U->cat2, 8, 32, n2);
  put(U->a3a, 0, 64, n3);
  put(U->a3b, 0, 64, n3);
  put(U->a2d, 0, 32, n2);
  put(U->a2b, 0, 32, n2);
  put(U->a1d, 0, 16, n1);
  put(U->u1, 0, 16, n1);
  cudaMemcpyAsync(tmp + o, U->g0, sizeof(float) * n1, cudaMemcpyDeviceToDevice, U->st);
  cudaMemcpyAsync(acts, tmp, sizeof(float) * need, cudaMemcpyDeviceToHost, U->st);
  if (train) {
    if ((r = backward(U, tmp))) {
      cudaStreamSynchronize(U->st);
      dfree(tmp);
      return r;
    }
    cudaMemcpyAsync(gz, tmp, sizeof(float) * need_g, cudaMemcpyDeviceToHost, U->st);
  }
  r = finish(U);
  cudaStreamSynchronize(U->st);
  dfree(tmp);
  return r;
}

}  // extern "C"
