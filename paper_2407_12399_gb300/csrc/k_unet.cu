// k_unet.cu -- kernels of the learned warm start: a 3-level 3D U-Net
// (channels 16/32/64, 3x3x3 convolutions, bf16 storage, fp32 accumulation)
// whose forward and backward passes run here.  The paper has no learned
// component; the network only proposes a starting field that the solver of
// Algorithm 1 then refines.
//
// Activation layout ("chunk planes"): a tensor of C channels on an
// (lz, ly, lx) grid is C/8 planes of lz*ly*lx voxels x 8 bf16 channels,
//   act[c / 8][z][y][x][c % 8],
// so one voxel's 8 channels of a plane are one 16-byte row.  A concatenated
// input is just more planes of the same buffer.
//
// Convolution (forward, and the data gradient as a convolution with the
// flipped, transposed kernel) is an implicit GEMM on the tcgen05 tensor
// cores: M = 128 output voxels (a run along x, or several short rows), N =
// output channels, K = 27 taps x input channels.  Per tap, TMA loads the
// 128 shifted input rows of every input plane straight from the chunk planes
// (out-of-grid rows arrive as zeros: the convolution's zero padding), which
// is exactly the no-swizzle K-major operand layout: 8-row x 16-byte core
// matrices, 128 B apart along M and 2 KiB apart along K.  The weights of a
// stage come in by one bulk copy, pre-packed in the same layout.  One thread
// issues the MMAs into a TMEM accumulator; all four warps read it back with
// tcgen05.ld for the epilogue (bias + ReLU or the ReLU mask of the data
// gradient, rounding to bf16).
//
// Weight gradients, pooling, upsampling, the 1x1 head, the loss and Adam are
// bandwidth-bound and run on the CUDA cores.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tsf_unet.cuh"

namespace tsf {
namespace unet {

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05, TMA, mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false after ~2^22 polls
// (seconds), so a kernel that would wait forever reports and returns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (between core matrices adjacent along K), stride byte offset
// (between core matrices adjacent along M or N), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void unpack8(const uint4& q, float* v) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
  }
}

__device__ __forceinline__ uint4 pack8(const float* v) {
  return make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                    pack_bf16x2(v[6], v[7]));
}

// ---------------------------------------------------------------------------
// Convolution as an implicit GEMM on tcgen05
// ---------------------------------------------------------------------------
// Shared memory per CTA: kStages x (A stage | B stage), then the barriers.
// A stage holds taps_per_stage x chunks K-chunks of 128 rows x 16 B; a B
// stage the same K-chunks of cout rows x 16 B.
__global__ void __launch_bounds__(128) k_conv_tc(const __grid_constant__ CUtensorMap in_map, ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t a_bytes = static_cast<uint32_t>(a.kchunks) * 2048u;
  const uint32_t b_bytes = static_cast<uint32_t>(a.kchunks) * static_cast<uint32_t>(a.cout) * 16u;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kConvStages * stage_bytes);
  uint64_t* empty = full + kConvStages;
  uint64_t* done = empty + kConvStages;
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(done + 1);
  int* s_abort = reinterpret_cast<int*>(s_taddr + 1);

  // tile of 128 rows: bx voxels along x times by rows along y, at one z
  const int tiles_x = (a.lx + a.bx - 1) / a.bx, tiles_y = (a.ly + a.by - 1) / a.by;
  int t = blockIdx.x;
  const int x0 = (t % tiles_x) * a.bx;
  t /= tiles_x;
  const int y0 = (t % tiles_y) * a.by;
  const int z0 = t / tiles_y;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kConvStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    s_abort[0] = 0;
    s_abort[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {  // TMEM accumulator: a.tmem_cols fp32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_taddr)),
                 "r"(static_cast<uint32_t>(a.tmem_cols))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_taddr;
  const int nst = a.nstages;

  if (warp == 0 && lane == 0) {
    // producer: per stage, the shifted input rows of its taps and its weights
    for (int s = 0; s < nst; ++s) {
      const int slot = s % kConvStages;
      if (s >= kConvStages) {
        if (!mbar_wait(&empty[slot], ((s / kConvStages) - 1) & 1)) {
          atomicOr(a.status, kUnetErrSpin);
          *reinterpret_cast<volatile int*>(s_abort) = 1;
          break;
        }
      }
      if (*reinterpret_cast<volatile int*>(s_abort)) break;
      uint8_t* sa = smem + slot * stage_bytes;
      mbar_expect_tx(&full[slot], stage_bytes);
      for (int q = 0; q < a.taps_per_stage; ++q) {
        const int tap = min(s * a.taps_per_stage + q, 26);  // a padding tap repeats tap 26 with zero weights
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        tma_load_5d(sa + q * a.chunks * 2048, &in_map, 0, x0 + dx - 1, y0 + dy - 1, z0 + dz - 1, 0, &full[slot]);
      }
      bulk_load(sa + a_bytes, a.wpack + static_cast<size_t>(s) * (b_bytes / 2), b_bytes, &full[slot]);
      s_abort[2] = s + 1;  // stages issued
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: K16 steps over the stage's K-chunks
    const uint32_t idesc = instr_desc(128, a.cout);
    for (int s = 0; s < nst; ++s) {
      const int slot = s % kConvStages;
      if (!mbar_wait(&full[slot], (s / kConvStages) & 1)) {
        atomicOr(a.status, kUnetErrSpin);
        *reinterpret_cast<volatile int*>(s_abort) = 1;
        break;
      }
      if (*reinterpret_cast<volatile int*>(s_abort)) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + slot * stage_bytes);
      const uint32_t sb = sa + a_bytes;
      for (int k = 0; k < a.kchunks / 2; ++k) {
        const uint64_t ad = smem_desc(sa + k * 4096u, 2048u, 128u);
        const uint64_t bd = smem_desc(sb + k * 2u * a.cout * 16u, a.cout * 16u, 128u);
        mma_bf16(taddr, ad, bd, idesc, (s > 0 || k > 0) ? 1u : 0u);
      }
      mma_commit(&empty[slot]);  // the slot is free once these MMAs have read it
    }
    mma_commit(done);  // arrives when every MMA issued above has completed
  }
  __syncwarp();

  // epilogue: one thread waits for the accumulator, then every row m = this
  // thread's TMEM lane
  if (threadIdx.x == 64) {
    bool ok = mbar_wait(done, 0);
    if (!ok) atomicOr(a.status, kUnetErrSpin);
    if (*reinterpret_cast<volatile int*>(s_abort)) ok = false;
    s_abort[1] = ok ? 1 : 0;
  }
  __syncthreads();
  const bool ok = s_abort[1] != 0;
  tc_fence_after();
  const int m = threadIdx.x;  // 0..127 = 32 * warp + lane
  const int x = x0 + m % a.bx, y = y0 + m / a.bx, z = z0;
  const bool inside = ok && x < a.lx && y < a.ly && z < a.lz;
  const size_t nv = static_cast<size_t>(a.lx) * a.ly * a.lz;
  const size_t vox = (static_cast<size_t>(z) * a.ly + y) * a.lx + x;
  for (int c8 = 0; c8 < a.cout / 8; ++c8) {
    float v[8];
    __syncwarp();
    tmem_ld8(taddr + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c8 * 8), v);  // warp-wide
    if (!inside) continue;
    if (a.mode == kConvForward) {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = fmaxf(v[i] + a.bias[c8 * 8 + i], 0.0f);
      const uint4 q = pack8(v);
      if (a.up) {  // nearest x2 upsampling: the voxel's 2x2x2 block of the fine grid
        const int fx = a.lx * 2, fy = a.ly * 2;
        const size_t fnv = nv * 8;
        uint4* base = reinterpret_cast<uint4*>(a.out) + (a.out_plane0 + c8) * fnv;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const size_t fv = (static_cast<size_t>(2 * z + (k >> 2)) * fy + (2 * y + ((k >> 1) & 1))) * fx + 2 * x + (k & 1);
          base[fv] = q;
        }
      } else {
        reinterpret_cast<uint4*>(a.out)[(a.out_plane0 + c8) * nv + vox] = q;
      }
    } else {  // data gradient, masked by the ReLU of the activation it flows into
      if (a.mask) {
        float mk[8];
        unpack8(reinterpret_cast<const uint4*>(a.mask)[(a.mask_plane0 + c8) * nv + vox], mk);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = mk[i] > 0.0f ? v[i] : 0.0f;
      }
      reinterpret_cast<uint4*>(a.out)[(a.out_plane0 + c8) * nv + vox] = pack8(v);
    }
  }
  // after an abort, wait (bounded) for the copies still in flight before the
  // shared memory they target is released
  if (threadIdx.x == 0 && !ok) {
    for (int s = max(0, s_abort[2] - kConvStages); s < s_abort[2]; ++s)
      mbar_wait(&full[s % kConvStages], (s / kConvStages) & 1);
  }
  tc_fence_before();
  __syncthreads();
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(static_cast<uint32_t>(a.tmem_cols))
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Bandwidth-bound layers on the CUDA cores
// ---------------------------------------------------------------------------
// Network input: plane 0 = (f, tau, 0, ..., 0) rounded to bf16.
__global__ void k_pack_input(const float* __restrict__ f, float tau, int64_t nv, uint4* __restrict__ x) {
  const int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (v >= nv) return;
  const float c[8] = {f[v], tau, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  x[v] = pack8(c);
}

// 2x2x2 average pooling of `planes` planes (fine grid lx, ly, lz).
__global__ void k_avgpool(const uint4* __restrict__ in, int in_plane0, int planes, int lx, int ly, int lz,
                          uint4* __restrict__ out) {
  const int cx = lx / 2, cy = ly / 2, cz = lz / 2;
  const int64_t cnv = static_cast<int64_t>(cx) * cy * cz, fnv = static_cast<int64_t>(lx) * ly * lz;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= cnv * planes) return;
  const int p = static_cast<int>(i / cnv);
  const int64_t v = i % cnv;
  const int x = static_cast<int>(v % cx), y = static_cast<int>((v / cx) % cy), z = static_cast<int>(v / (static_cast<int64_t>(cx) * cy));
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < 8; ++k) {
    const int64_t fv = (static_cast<int64_t>(2 * z + (k >> 2)) * ly + 2 * y + ((k >> 1) & 1)) * lx + 2 * x + (k & 1);
    float t[8];
    unpack8(in[(in_plane0 + p) * fnv + fv], t);
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += t[c];
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] *= 0.125f;
  out[p * cnv + v] = pack8(acc);
}

// Backward of "upsample, then concatenate": the gradient of the coarse
// activation is the sum of its 2x2x2 fine gradients, masked by its ReLU.
// g: fine gradient planes [g_plane0, g_plane0 + planes); act: the coarse
// activation (read through the upsampled copy: any of its 8 fine voxels).
__global__ void k_upsample_back(const uint4* __restrict__ g, int g_plane0, int planes, int lx, int ly, int lz,
                                const uint4* __restrict__ act_up, int act_plane0, uint4* __restrict__ out) {
  const int cx = lx / 2, cy = ly / 2, cz = lz / 2;
  const int64_t cnv = static_cast<int64_t>(cx) * cy * cz, fnv = static_cast<int64_t>(lx) * ly * lz;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= cnv * planes) return;
  const int p = static_cast<int>(i / cnv);
  const int64_t v = i % cnv;
  const int x = static_cast<int>(v % cx), y = static_cast<int>((v / cx) % cy), z = static_cast<int>(v / (static_cast<int64_t>(cx) * cy));
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t fv0 = 0;
  for (int k = 0; k < 8; ++k) {
    const int64_t fv = (static_cast<int64_t>(2 * z + (k >> 2)) * ly + 2 * y + ((k >> 1) & 1)) * lx + 2 * x + (k & 1);
    if (k == 0) fv0 = fv;
    float t[8];
    unpack8(g[(g_plane0 + p) * fnv + fv], t);
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += t[c];
  }
  float a[8];
  unpack8(act_up[(act_plane0 + p) * fnv + fv0], a);
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = a[c] > 0.0f ? acc[c] : 0.0f;
  out[p * cnv + v] = pack8(acc);
}

// Gradient of a skip activation s (fine grid): its share from the
// concatenation plus the average-pooling backward of the coarse gradient gp,
// masked by s's ReLU.
__global__ void k_skip_back(const uint4* __restrict__ gs, int gs_plane0, const uint4* __restrict__ gp,
                            const uint4* __restrict__ s, int s_plane0, int planes, int lx, int ly, int lz,
                            uint4* __restrict__ out) {
  const int64_t fnv = static_cast<int64_t>(lx) * ly * lz;
  const int cx = lx / 2, cy = ly / 2;
  const int64_t cnv = fnv / 8;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= fnv * planes) return;
  const int p = static_cast<int>(i / fnv);
  const int64_t v = i % fnv;
  const int x = static_cast<int>(v % lx), y = static_cast<int>((v / lx) % ly), z = static_cast<int>(v / (static_cast<int64_t>(lx) * ly));
  const int64_t cv = (static_cast<int64_t>(z / 2) * cy + y / 2) * cx + x / 2;
  float a[8], b[8], m[8];
  unpack8(gs[(gs_plane0 + p) * fnv + v], a);
  unpack8(gp[p * cnv + cv], b);
  unpack8(s[(s_plane0 + p) * fnv + v], m);
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = m[c] > 0.0f ? a[c] + b[c] * 0.125f : 0.0f;
  out[p * fnv + v] = pack8(a);
}

// Head, forward: g0 = f + bf16(sum_c u1[c] w[c] + b) (two planes of u1);
// hw holds the 16 weights and then the bias.
__global__ void k_head_forward(const uint4* __restrict__ u1, const float* __restrict__ hw, int64_t nv,
                               const float* __restrict__ f, float* __restrict__ g0) {
  const int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (v >= nv) return;
  const float hb = hw[16];
  float a[8], b[8];
  unpack8(u1[v], a);
  unpack8(u1[nv + v], b);
  float r = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) r = fmaf(a[c], hw[c], r);
#pragma unroll
  for (int c = 0; c < 8; ++c) r = fmaf(b[c], hw[8 + c], r);
  r = __bfloat162float(__float2bfloat16_rn(r + hb));
  g0[v] = f[v] + r;
}

// Head, backward for the loss mean((g0 - g)^2): per voxel gg = 2 (g0 - g) / nv;
// the u1 gradient gg * w masked by u1's ReLU; block partial sums (fp64) of
// the loss, of gg and of gg * u1[c] (the head's bias and weight gradients).
__global__ void __launch_bounds__(256) k_head_backward(const uint4* __restrict__ u1, const float* __restrict__ hw,
                                                       int64_t nv, const float* __restrict__ f,
                                                       const float* __restrict__ g, uint4* __restrict__ gz,
                                                       double* __restrict__ partial) {
  __shared__ double red[18][8];
  const float hb = hw[16];
  const int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  double acc[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) acc[k] = 0.0;
  if (v < nv) {
    float a[16];
    unpack8(u1[v], a);
    unpack8(u1[nv + v], a + 8);
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < 16; ++c) r = fmaf(a[c], hw[c], r);
    r = __bfloat162float(__float2bfloat16_rn(r + hb));
    const float d = (f[v] + r) - g[v];
    const float gg = 2.0f * d / static_cast<float>(nv);
    acc[0] = static_cast<double>(d) * d;
    acc[1] = gg;
    float o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      acc[2 + c] = static_cast<double>(gg) * a[c];
      o[c] = a[c] > 0.0f ? gg * hw[c] : 0.0f;
    }
    gz[v] = pack8(o);
    gz[nv + v] = pack8(o + 8);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    double x = acc[k];
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < 18) {
    double x = 0.0;
    for (int i = 0; i < 8; ++i) x += red[threadIdx.x][i];
    partial[static_cast<int64_t>(blockIdx.x) * 18 + threadIdx.x] = x;
  }
}

// Sums the head's block partials in block order: out[0] = loss (mean),
// grad[hw_off + c] = sum gg u1[c], grad[hb_off] = sum gg.
__global__ void k_head_reduce(const double* __restrict__ partial, int nblocks, int64_t nv, double* __restrict__ loss,
                              float* __restrict__ grad, int64_t hw_off, int64_t hb_off) {
  const int k = threadIdx.x;
  if (k >= 18) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[static_cast<int64_t>(b) * 18 + k];
  if (k == 0) *loss = s / static_cast<double>(nv);
  else if (k == 1) grad[hb_off] = static_cast<float>(s);
  else grad[hw_off + (k - 2)] = static_cast<float>(s);
}

// Weight gradient of one convolution: gw[o][c][tap] = sum over voxels p of
// gz[o][p] x[c][p + tap - 1] (zero outside the grid), gb[o] = sum gz[o][p].
// Block (tap, chunk of kWgV voxels in linear order); each thread owns a
// 4 (o) x 4 (c) register tile and a share of the voxels; partial sums per
// block, reduced in block order by k_wgrad_reduce (deterministic).
constexpr int kWgV = 64;     // voxels staged in shared memory at a time
constexpr int kWgChunk = 1024;  // voxels per block

__global__ void __launch_bounds__(256) k_wgrad(const uint4* __restrict__ x, int x_plane0, int cin,
                                               const uint4* __restrict__ gz, int cout, int lx, int ly, int lz,
                                               float* __restrict__ partial) {
  extern __shared__ float wsm[];
  float* sg = wsm;                    // [cout][kWgV]
  float* sx = wsm + cout * kWgV;      // [cin][kWgV]
  float* sred = sx + cin * kWgV;      // reduction across voxel groups
  const int tap = blockIdx.y;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int64_t nv = static_cast<int64_t>(lx) * ly * lz;
  const int64_t v0 = static_cast<int64_t>(blockIdx.x) * kWgChunk;
  const int to = cout / 4, tc = cin / 4, ntile = to * tc;
  const int groups = max(1, 256 / ntile);  // voxel groups sharing the tiles
  const int tid = threadIdx.x;
  const int tile = tid % ntile, grp = tid / ntile;
  const bool active = tid < ntile * groups;
  const int o0 = (tile / tc) * 4, c0 = (tile % tc) * 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int64_t vb = v0; vb < v0 + kWgChunk && vb < nv; vb += kWgV) {
    __syncthreads();
    // stage gz (cout planes) and the tap-shifted x (cin planes) as fp32
    for (int i = tid; i < (cout / 8) * kWgV; i += 256) {
      const int p = i / kWgV, k = i % kWgV;
      const int64_t v = vb + k;
      float t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (v < nv) unpack8(gz[p * nv + v], t);
#pragma unroll
      for (int c = 0; c < 8; ++c) sg[(p * 8 + c) * kWgV + k] = t[c];
    }
    for (int i = tid; i < (cin / 8) * kWgV; i += 256) {
      const int p = i / kWgV, k = i % kWgV;
      const int64_t v = vb + k;
      float t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (v < nv) {
        const int vx = static_cast<int>(v % lx) + dx, vy = static_cast<int>((v / lx) % ly) + dy,
                  vz = static_cast<int>(v / (static_cast<int64_t>(lx) * ly)) + dz;
        if (vx >= 0 && vx < lx && vy >= 0 && vy < ly && vz >= 0 && vz < lz)
          unpack8(x[(x_plane0 + p) * nv + (static_cast<int64_t>(vz) * ly + vy) * lx + vx], t);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) sx[(p * 8 + c) * kWgV + k] = t[c];
    }
    __syncthreads();
    if (active) {
      for (int k = grp; k < kWgV; k += groups) {
        float go[4], xc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) go[i] = sg[(o0 + i) * kWgV + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) xc[j] = sx[(c0 + j) * kWgV + k];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(go[i], xc[j], acc[i][j]);
      }
    }
  }
  // combine the voxel groups (fixed order), then write the block's partial
  __syncthreads();
  float* out = partial + (static_cast<int64_t>(tap) * gridDim.x + blockIdx.x) * cout * cin;
  for (int g = 0; g < groups; ++g) {
    if (active && grp == g) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float* p = &sred[(o0 + i) * cin + c0 + j];
          *p = (g == 0 ? 0.0f : *p) + acc[i][j];
        }
    }
    __syncthreads();
  }
  for (int i = tid; i < cout * cin; i += 256) out[i] = sred[i];
}

// gw in the reference layout (cout, cin_real, 3, 3, 3) = sum over blocks of
// the partials, in block order.
__global__ void k_wgrad_reduce(const float* __restrict__ partial, int nblk, int cout, int cin, int cin_real,
                               float* __restrict__ gw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 27 * cout * cin_real
  if (i >= 27 * cout * cin_real) return;
  const int tap = i % 27, c = (i / 27) % cin_real, o = i / (27 * cin_real);
  const float* p = partial + static_cast<int64_t>(tap) * nblk * cout * cin + o * cin + c;
  float s = 0.0f;
  for (int b = 0; b < nblk; ++b) s += p[static_cast<int64_t>(b) * cout * cin];
  gw[i] = s;
}

// gb[o] = sum over voxels of gz[o]: block partials, then an ordered sum.
__global__ void __launch_bounds__(256) k_bias_partial(const uint4* __restrict__ gz, int cout, int64_t nv,
                                                      float* __restrict__ partial) {
  __shared__ float red[8][96];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t v0 = static_cast<int64_t>(blockIdx.x) * 2048;
  for (int p = 0; p < cout / 8; ++p) {
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t v = v0 + threadIdx.x; v < v0 + 2048 && v < nv; v += 256) {
      float t[8];
      unpack8(gz[p * nv + v], t);
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] += t[c];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float x = acc[c];
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
      if (lane == 0) red[w][p * 8 + c] = x;
    }
  }
  __syncthreads();
  if (threadIdx.x < cout) {
    float s = 0.0f;
    for (int i = 0; i < 8; ++i) s += red[i][threadIdx.x];
    partial[static_cast<int64_t>(blockIdx.x) * cout + threadIdx.x] = s;
  }
}

__global__ void k_bias_reduce(const float* __restrict__ partial, int nblk, int cout, float* __restrict__ gb) {
  const int o = threadIdx.x;
  if (o >= cout) return;
  float s = 0.0f;
  for (int b = 0; b < nblk; ++b) s += partial[static_cast<int64_t>(b) * cout + o];
  gb[o] = s;
}

// Weights of one layer from the fp32 master copy (reference layout
// (cout, cin_real, 3, 3, 3)) into the stage-packed bf16 B operand:
// pack[stage][kchunk][o][8], kchunk over (tap in stage, input chunk).  The
// data-gradient packing transposes and flips: B[o'][c'][tap] =
// w[c'][o'][26 - tap] (o' over the forward inputs, c' over its outputs).
__global__ void k_pack_weights(const float* __restrict__ w, int cout_f, int cin_real, int cin_pad, int taps_per_stage,
                               int nstages, int transpose, __nv_bfloat16* __restrict__ pack) {
  const int n_out = transpose ? cin_pad : cout_f;   // N of the GEMM
  const int n_in = transpose ? cout_f : cin_pad;    // input channels of the GEMM
  const int chunks = n_in / 8;
  const int kchunks = taps_per_stage * chunks;
  const int64_t total = static_cast<int64_t>(nstages) * kchunks * n_out * 8;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= total) return;
  const int e = static_cast<int>(i % 8);
  const int o = static_cast<int>((i / 8) % n_out);
  const int kc = static_cast<int>((i / (8 * n_out)) % kchunks);
  const int s = static_cast<int>(i / (static_cast<int64_t>(8) * n_out * kchunks));
  const int tap = s * taps_per_stage + kc / chunks;
  const int ci = (kc % chunks) * 8 + e;
  float val = 0.0f;
  if (tap < 27) {
    if (!transpose) {
      if (ci < cin_real) val = w[(static_cast<int64_t>(o) * cin_real + ci) * 27 + tap];
    } else {  // GEMM output o = forward input channel, GEMM input ci = forward output channel
      if (o < cin_real) val = w[(static_cast<int64_t>(ci) * cin_real + o) * 27 + (26 - tap)];
    }
  }
  pack[i] = __float2bfloat16_rn(val);
}

// Biases and head weights rounded to bf16 (kept as fp32 values).
__global__ void k_round_bf16(const float* __restrict__ in, int64_t n, float* __restrict__ out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = __bfloat162float(__float2bfloat16_rn(in[i]));
}

// Adam (Kingma & Ba, Algorithm 1) on the fp32 master parameters; bc1 and bc2
// are 1 - beta1^t and 1 - beta2^t.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float beta1, float beta2, float eps, float bc1,
                       float bc2) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / bc1, vh = vi / bc2;
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Planes (bf16) -> fp32 in the reference layout (C, z, y, x), `c_real`
// channels of the planes starting at plane0.
__global__ void k_unpack_planes(const uint4* __restrict__ in, int plane0, int c_real, int64_t nv,
                                float* __restrict__ out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= nv * c_real) return;
  const int c = static_cast<int>(i / nv);
  const int64_t v = i % nv;
  float t[8];
  unpack8(in[(plane0 + c / 8) * nv + v], t);
  out[i] = t[c % 8];
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
namespace {
// cuTensorMapEncodeTiled, looked up through the runtime (no link to libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
bool g_attr_set[64] = {};
}  // namespace

int encode_planes_map(CUtensorMap* map, const void* base, int lx, int ly, int lz, int chunks, int bx, int by) {
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const uint64_t nv = static_cast<uint64_t>(lx) * ly * lz;
  cuuint64_t dims[5] = {8, static_cast<cuuint64_t>(lx), static_cast<cuuint64_t>(ly), static_cast<cuuint64_t>(lz),
                        static_cast<cuuint64_t>(chunks)};
  cuuint64_t strides[4] = {16, 16ull * lx, 16ull * lx * ly, 16ull * nv};
  cuuint32_t box[5] = {8, static_cast<cuuint32_t>(bx), static_cast<cuuint32_t>(by), 1,
                       static_cast<cuuint32_t>(chunks)};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

void tile_shape(int lx, int& bx, int& by) {
  if (lx >= 128 || 128 % lx != 0) {
    bx = 128;
    by = 1;
  } else {
    bx = lx;
    by = 128 / lx;
  }
}

// Stages, barriers and alignment slack, plus a guard region that keeps every
// address an operand descriptor of a stage can span (up to 32 KiB past the
// start of its A or B tile) inside the allocation.
size_t conv_smem_bytes(int kchunks, int cout) {
  const size_t stage = static_cast<size_t>(kchunks) * 2048 + static_cast<size_t>(kchunks) * cout * 16;
  return 1024 + kConvStages * stage + (2 * kConvStages + 1) * 8 + 32 + 40 * 1024;
}

int launch_conv(const ConvArgs& a0, const void* in_planes, int in_chunks, cudaStream_t st) {
  ConvArgs a = a0;
  a.chunks = in_chunks;
  a.taps_per_stage = in_chunks == 1 ? 2 : 1;
  a.kchunks = a.taps_per_stage * in_chunks;
  a.nstages = (27 + a.taps_per_stage - 1) / a.taps_per_stage;
  a.tmem_cols = a.cout <= 32 ? 32 : (a.cout <= 64 ? 64 : 128);
  if (a.cout % 16 != 0 || a.cout > 128 || in_chunks > 12) return -1;
  tile_shape(a.lx, a.bx, a.by);
  CUtensorMap map;
  if (encode_planes_map(&map, in_planes, a.lx, a.ly, a.lz, in_chunks, a.bx, a.by) != 0) return -2;
  const size_t smem = conv_smem_bytes(a.kchunks, a.cout);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !g_attr_set[dev]) {
    cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kConvMaxSmem));
    g_attr_set[dev] = true;
  }
  if (smem > kConvMaxSmem) return -3;
  const int tiles = ((a.lx + a.bx - 1) / a.bx) * ((a.ly + a.by - 1) / a.by) * a.lz;
  k_conv_tc<<<tiles, 128, smem, st>>>(map, a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -4;
}

void launch_pack_input(const float* f, float tau, int64_t nv, void* x, cudaStream_t st) {
  k_pack_input<<<static_cast<unsigned>((nv + 255) / 256), 256, 0, st>>>(f, tau, nv, static_cast<uint4*>(x));
}

void launch_avgpool(const void* in, int in_plane0, int planes, int lx, int ly, int lz, void* out, cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(lx / 2) * (ly / 2) * (lz / 2) * planes;
  k_avgpool<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(static_cast<const uint4*>(in), in_plane0, planes,
                                                                    lx, ly, lz, static_cast<uint4*>(out));
}

void launch_upsample_back(const void* g, int g_plane0, int planes, int lx, int ly, int lz, const void* act_up,
                          int act_plane0, void* out, cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(lx / 2) * (ly / 2) * (lz / 2) * planes;
  k_upsample_back<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(
      static_cast<const uint4*>(g), g_plane0, planes, lx, ly, lz, static_cast<const uint4*>(act_up), act_plane0,
      static_cast<uint4*>(out));
}

void launch_skip_back(const void* gs, int gs_plane0, const void* gp, const void* s, int s_plane0, int planes, int lx,
                      int ly, int lz, void* out, cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(lx) * ly * lz * planes;
  k_skip_back<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(
      static_cast<const uint4*>(gs), gs_plane0, static_cast<const uint4*>(gp), static_cast<const uint4*>(s), s_plane0,
      planes, lx, ly, lz, static_cast<uint4*>(out));
}

void launch_head_forward(const void* u1, const float* hw, int64_t nv, const float* f, float* g0, cudaStream_t st) {
  k_head_forward<<<static_cast<unsigned>((nv + 255) / 256), 256, 0, st>>>(static_cast<const uint4*>(u1), hw, nv, f,
                                                                         g0);
}

int head_blocks(int64_t nv) { return static_cast<int>((nv + 255) / 256); }

void launch_head_backward(const void* u1, const float* hw, int64_t nv, const float* f, const float* g, void* gz,
                          double* partial, double* loss, float* grad, int64_t hw_off, int64_t hb_off, cudaStream_t st) {
  const int nb = head_blocks(nv);
  k_head_backward<<<nb, 256, 0, st>>>(static_cast<const uint4*>(u1), hw, nv, f, g, static_cast<uint4*>(gz), partial);
  k_head_reduce<<<1, 32, 0, st>>>(partial, nb, nv, loss, grad, hw_off, hb_off);
}

int64_t wgrad_partial_floats(int64_t nv, int cout, int cin) {
  const int64_t nblk = (nv + kWgChunk - 1) / kWgChunk;
  return 27 * nblk * cout * cin;
}

int64_t bias_partial_floats(int64_t nv, int cout) { return ((nv + 2047) / 2048) * cout; }

void launch_wgrad(const void* x, int x_plane0, int cin, int cin_real, const void* gz, int cout, int lx, int ly, int lz,
                  float* partial, float* gw, float* bpartial, float* gb, cudaStream_t st) {
  const int64_t nv = static_cast<int64_t>(lx) * ly * lz;
  const int nblk = static_cast<int>((nv + kWgChunk - 1) / kWgChunk);
  const size_t smem = (static_cast<size_t>(cout + cin) * kWgV + static_cast<size_t>(cout) * cin) * sizeof(float);
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr[dev] = true;
  }
  k_wgrad<<<dim3(nblk, 27), 256, smem, st>>>(static_cast<const uint4*>(x), x_plane0, cin,
                                             static_cast<const uint4*>(gz), cout, lx, ly, lz, partial);
  const int n = 27 * cout * cin_real;
  k_wgrad_reduce<<<(n + 255) / 256, 256, 0, st>>>(partial, nblk, cout, cin, cin_real, gw);
  const int nb = static_cast<int>((nv + 2047) / 2048);
  k_bias_partial<<<nb, 256, 0, st>>>(static_cast<const uint4*>(gz), cout, nv, bpartial);
  k_bias_reduce<<<1, 128, 0, st>>>(bpartial, nb, cout, gb);
}

void launch_pack_weights(const float* w, int cout_f, int cin_real, int cin_pad, int transpose, void* pack,
                         cudaStream_t st) {
  const int n_in = transpose ? cout_f : cin_pad;
  const int chunks = n_in / 8;
  const int tps = chunks == 1 ? 2 : 1;
  const int nstages = (27 + tps - 1) / tps;
  const int n_out = transpose ? cin_pad : cout_f;
  const int64_t total = static_cast<int64_t>(nstages) * tps * chunks * n_out * 8;
  k_pack_weights<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(
      w, cout_f, cin_real, cin_pad, tps, nstages, transpose, static_cast<__nv_bfloat16*>(pack));
}

int64_t pack_elems(int cout_f, int cin_pad, int transpose) {
  const int n_in = transpose ? cout_f : cin_pad;
  const int chunks = n_in / 8;
  const int tps = chunks == 1 ? 2 : 1;
  const int nstages = (27 + tps - 1) / tps;
  const int n_out = transpose ? cin_pad : cout_f;
  return static_cast<int64_t>(nstages) * tps * chunks * n_out * 8;
}

void launch_round_bf16(const float* in, int64_t n, float* out, cudaStream_t st) {
  k_round_bf16<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(in, n, out);
}

void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                 float eps, float bc1, float bc2, cudaStream_t st) {
  k_adam<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, lr, beta1, beta2, eps, bc1, bc2);
}

void launch_unpack_planes(const void* in, int plane0, int c_real, int64_t nv, float* out, cudaStream_t st) {
  const int64_t n = nv * c_real;
  k_unpack_planes<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(static_cast<const uint4*>(in), plane0,
                                                                         c_real, nv, out);
}

}  // namespace unet
}  // namespace tsf
