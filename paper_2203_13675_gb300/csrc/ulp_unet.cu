// ulp_unet.cu -- learned preconditioner: a four-level U-Net evaluated as
// s = rho * N_theta(r / rho, U, V) inside flexible CG, and its training.
//
// Network (channels 16/32/64/128, 3x3 convolutions with ReLU, 2x2 average
// pooling, nearest-neighbour upsampling, a linear 1x1 head):
//   e0: 3->16 at H x W      e1: 16->32 at H/2     e2: 32->64 at H/4     b3: 64->128 at H/8
//   d2: [a2 | up(b3)] 192->64 at H/4   d1: [a1 | up(d2)] 96->32 at H/2   d0: [a0 | up(d1)] 48->16 at H
//   head: y = w_h . d0 + b_h
// Activations are NHWC BF16.  The concatenated decoder inputs are never
// assembled by a copy: each level's buffer cat_l = [a_l | up(next)] is written
// in place, a_l by the encoder convolution's epilogue at channel offset 0 and
// up(next) by the lower level's epilogue, which writes every output pixel to
// its 2x2 block at the upper channel offset.
//
// Every 3x3 convolution is an implicit GEMM on the 5th-generation tensor
// cores: a CTA owns 128 output pixels (M) and all Cout channels (N); K = 9 Cin
// runs over taps and 16-channel chunks.  For tap (dy, dx) and chunk c the A
// tile is the TMA box {16 ch, bw, bh, 1} at (16c, x0 + dx - 1, y0 + dy - 1, b),
// 32-byte swizzled; coordinates outside the image read zeros, which is the
// convolution's zero padding.  The B tile is the weight box {16, Cout} of
// [Cout][9 Cin] BF16 weights.  One K = 16 MMA per stage, a 6-stage ring, the
// FP32 accumulator in tensor memory; bias, ReLU and the BF16 store are fused
// into the epilogue.  The input gradient of a convolution is the same kernel
// on the output gradient with the weights transposed and the taps reversed;
// the weight gradient is an FP32 CUDA-core reduction over pixels.  Every
// reduction runs in a fixed order, so results do not depend on scheduling.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ulp_host.h"
#include "ulp_tc.cuh"

namespace ulp {
namespace unet {

using bf16 = __nv_bfloat16;

constexpr int kNL = 7;
enum { E0 = 0, E1, E2, B3, D2, D1, D0 };
constexpr int kCin[kNL] = {3, 16, 32, 64, 192, 96, 48};
constexpr int kCinPad[kNL] = {16, 16, 32, 64, 192, 96, 48};
constexpr int kCout[kNL] = {16, 32, 64, 128, 64, 32, 16};
constexpr int kMaxBatch = 64;
constexpr int kPartRows = 2048;            // weight-gradient partial slots (x 2320 floats)
constexpr int kPartCols = 16 * 16 * 9 + 16;

struct Offsets {
  long long w[kNL], b[kNL], hw, hb, n;
};
static Offsets offsets() {
  Offsets o{};
  long long k = 0;
  for (int l = 0; l < kNL; ++l) {
    o.w[l] = k;
    k += (long long)kCout[l] * kCin[l] * 9;
    o.b[l] = k;
    k += kCout[l];
  }
  o.hw = k;
  o.hb = k + 16;
  o.n = k + 17;
  return o;
}

struct Offs {
  long long o[kMaxBatch];
};

// ------------------------------------------------------------------ convolution
constexpr int kCStages = 6;
constexpr int kATile = 128 * 32;  // 128 pixels x 16 channels x 2 bytes

struct ConvArgs {
  int H, W, Cin, Cout, bw, bh, tiles_x, tiles_img, tcols;
  const float* bias;
  int relu;
  bf16* y;
  int ystride, yoff, up;
  const int* skip;
  int* err;
};

static int conv_stage_bytes(int Cout) { return kATile + ((Cout * 32 + 1023) & ~1023); }
static int conv_smem(int Cout) { return kCStages * conv_stage_bytes(Cout) + 1024 + 256; }

__global__ void __launch_bounds__(128) k_conv3x3(const __grid_constant__ CUtensorMap tx,
                                                 const __grid_constant__ CUtensorMap tw, ConvArgs a) {
  if (a.skip && *(volatile const int*)a.skip) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int stage = kATile + ((a.Cout * 32 + 1023) & ~1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kCStages * stage);
  uint64_t* empty = full + kCStages;
  uint64_t* done = empty + kCStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x / a.tiles_img, tt = blockIdx.x - b * a.tiles_img;
  const int y0 = (tt / a.tiles_x) * a.bh, x0 = (tt % a.tiles_x) * a.bw;
  const int nch = a.Cin >> 4, nk = 9 * nch;
  const uint32_t idesc = idesc_bf16(128, a.Cout);
  const uint32_t btile = (uint32_t)a.Cout * 32u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kCStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    for (int k = 0; k < nk; ++k) {
      const int s = k % kCStages, u = k / kCStages;
      if (u > 0 && !mbar_wait(empty + s, (u - 1) & 1, a.err)) break;
      const int tap = k / nch, c = k - tap * nch;
      const int dy = tap / 3, dx = tap - 3 * dy;
      unsigned char* sa = base + s * stage;
      mbar_expect_tx(full + s, (uint32_t)kATile + btile);
      tma_load_4d(sa, &tx, full + s, c * 16, x0 + dx - 1, y0 + dy - 1, b);
      tma_load_2d(sa + kATile, &tw, full + s, tap * a.Cin + c * 16, 0);
    }
  } else if (warp == 1 && lane == 0) {
    for (int k = 0; k < nk; ++k) {
      const int s = k % kCStages, u = k / kCStages;
      if (!mbar_wait(full + s, u & 1, a.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned char* sa = base + s * stage;
      mma_bf16(tmem, sw32_desc(sa), sw32_desc(sa + kATile), idesc, k != 0);
      mma_commit(empty + s);
    }
    mma_commit(done);
  }
  __syncwarp();

  const bool ready = __all_sync(0xffffffffu, mbar_wait(done, 0, a.err));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready) {
    const int m = warp * 32 + lane;
    const int py = y0 + m / a.bw, px = x0 + (m % a.bw);
#pragma unroll 1
    for (int c = 0; c < (a.Cout >> 4); ++c) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
      __align__(16) bf16 o[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        float t = v[q] + (a.bias ? __ldg(a.bias + c * 16 + q) : 0.f);
        if (a.relu) t = fmaxf(t, 0.f);
        o[q] = __float2bfloat16_rn(t);
      }
      const uint4 lo = reinterpret_cast<const uint4*>(o)[0], hi = reinterpret_cast<const uint4*>(o)[1];
      if (!a.up) {
        uint4* dst = reinterpret_cast<uint4*>(a.y + ((size_t)(b * a.H + py) * a.W + px) * a.ystride + a.yoff + c * 16);
        dst[0] = lo;
        dst[1] = hi;
      } else {
        const int H2 = 2 * a.H, W2 = 2 * a.W;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int yy = 2 * py + (e >> 1), xx = 2 * px + (e & 1);
          uint4* dst = reinterpret_cast<uint4*>(a.y + ((size_t)(b * H2 + yy) * W2 + xx) * a.ystride + a.yoff + c * 16);
          dst[0] = lo;
          dst[1] = hi;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tcols));
}

// y = act(conv3x3(x, w) + bias): x [B][H][W][Cin], w [Cout][9][Cin], y written at
// channel offset yoff of a destination with ystride channels per pixel, either
// at (H, W) or (up) replicated to the 2x2 blocks of a (2H, 2W) destination.
static cudaError_t conv3x3(const bf16* x, int B, int H, int W, int Cin, const bf16* w, int Cout, const float* bias,
                           int relu, bf16* y, int ystride, int yoff, int up, const int* skip, int* err,
                           cudaStream_t st) {
  int bw = W & -W;
  if (bw > 128) bw = 128;
  const int bh = 128 / bw;
  if (Cin % 16 || Cout % 16 || Cout < 16 || Cout > 256 || B < 1 || B > 65535 || bh > H || H % bh || W % bw ||
      ystride % 16 || yoff % 16 || yoff + Cout > ystride)
    return cudaErrorInvalidValue;
  PFN_encodeTiled fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  CUtensorMap tx, tw;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t str[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)Cin * 2 * W, (cuuint64_t)Cin * 2 * W * H};
    const cuuint32_t box[4] = {16, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (fn(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x), dims, str, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)9 * Cin, (cuuint64_t)Cout};
    const cuuint64_t str[1] = {(cuuint64_t)9 * Cin * 2};
    const cuuint32_t box[2] = {16, (cuuint32_t)Cout};
    const cuuint32_t es[2] = {1, 1};
    if (fn(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(w), dims, str, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  int tcols = 32;
  while (tcols < Cout) tcols <<= 1;
  ConvArgs a{H, W, Cin, Cout, bw, bh, W / bw, (H / bh) * (W / bw), tcols, bias, relu, y, ystride, yoff, up, skip, err};
  const long long grid = (long long)B * a.tiles_img;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_conv3x3<<<(unsigned)grid, 128, conv_smem(Cout), st>>>(tx, tw, a);
  return cudaGetLastError();
}


// ------------------------------------------------------------------ elementwise kernels
__device__ __forceinline__ void unpack8(uint4 u, float (&f)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 t = __bfloat1622float2(h[k]);
    f[2 * k] = t.x;
    f[2 * k + 1] = t.y;
  }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
  return u;
}
__device__ __forceinline__ bool skipped(const int* skip) { return skip && *(volatile const int*)skip; }

#define GRID_STRIDE(t, n) for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (n); t += (size_t)gridDim.x * blockDim.x)

// 2x2 average pool of channels [0, C) of a buffer with Cs channels per pixel -> [B][H/2][W/2][C]
__global__ void k_pool2(const bf16* __restrict__ in, int Cs, int C, int B, int H, int W, bf16* __restrict__ out,
                        const int* skip) {
  if (skipped(skip)) return;
  const int Ho = H / 2, Wo = W / 2, G = C / 8;
  const size_t n = (size_t)B * Ho * Wo * G;
  GRID_STRIDE(t, n) {
    const int g = (int)(t % G);
    const size_t q = t / G;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), b = (int)(q / ((size_t)Wo * Ho));
    const bf16* p = in + ((size_t)(b * H + 2 * yo) * W + 2 * xo) * Cs + 8 * g;
    float f0[8], f1[8], f2[8], f3[8], o[8];
    unpack8(*reinterpret_cast<const uint4*>(p), f0);
    unpack8(*reinterpret_cast<const uint4*>(p + Cs), f1);
    unpack8(*reinterpret_cast<const uint4*>(p + (size_t)W * Cs), f2);
    unpack8(*reinterpret_cast<const uint4*>(p + (size_t)W * Cs + Cs), f3);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = 0.25f * ((f0[k] + f1[k]) + (f2[k] + f3[k]));
    *reinterpret_cast<uint4*>(out + q * C + 8 * g) = pack8(o);
  }
}

// gradient through up(): out[q][c] = (sum of the 2x2 block of dcat[.][coff + c]) * (cat[2q][coff + c] > 0)
__global__ void k_upsum_gate(const bf16* __restrict__ dcat, const bf16* __restrict__ cat, int Ctot, int coff, int C,
                             int B, int Hl, int Wl, bf16* __restrict__ out) {
  const int G = C / 8, H = 2 * Hl, W = 2 * Wl;
  const size_t n = (size_t)B * Hl * Wl * G;
  GRID_STRIDE(t, n) {
    const int g = (int)(t % G);
    const size_t q = t / G;
    const int xo = (int)(q % Wl), yo = (int)((q / Wl) % Hl), b = (int)(q / ((size_t)Wl * Hl));
    const size_t p00 = ((size_t)(b * H + 2 * yo) * W + 2 * xo) * Ctot + coff + 8 * g;
    float f0[8], f1[8], f2[8], f3[8], gt[8], o[8];
    unpack8(*reinterpret_cast<const uint4*>(dcat + p00), f0);
    unpack8(*reinterpret_cast<const uint4*>(dcat + p00 + Ctot), f1);
    unpack8(*reinterpret_cast<const uint4*>(dcat + p00 + (size_t)W * Ctot), f2);
    unpack8(*reinterpret_cast<const uint4*>(dcat + p00 + (size_t)W * Ctot + Ctot), f3);
    unpack8(*reinterpret_cast<const uint4*>(cat + p00), gt);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = gt[k] > 0.f ? (f0[k] + f1[k]) + (f2[k] + f3[k]) : 0.f;
    *reinterpret_cast<uint4*>(out + q * C + 8 * g) = pack8(o);
  }
}

// encoder gradient: out[p][c] = (dcat[p][c] + dlow[p/2][c] / 4) * (cat[p][c] > 0), c < C
__global__ void k_merge_gate(const bf16* __restrict__ dcat, const bf16* __restrict__ cat, int Ctot, int C,
                             const bf16* __restrict__ dlow, int B, int H, int W, bf16* __restrict__ out) {
  const int G = C / 8;
  const size_t n = (size_t)B * H * W * G;
  GRID_STRIDE(t, n) {
    const int g = (int)(t % G);
    const size_t q = t / G;
    const int x = (int)(q % W), y = (int)((q / W) % H), b = (int)(q / ((size_t)W * H));
    float f[8], gt[8], l[8] = {0, 0, 0, 0, 0, 0, 0, 0}, o[8];
    unpack8(*reinterpret_cast<const uint4*>(dcat + q * Ctot + 8 * g), f);
    unpack8(*reinterpret_cast<const uint4*>(cat + q * Ctot + 8 * g), gt);
    if (dlow)
      unpack8(*reinterpret_cast<const uint4*>(dlow + ((size_t)(b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + 8 * g), l);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = gt[k] > 0.f ? f[k] + 0.25f * l[k] : 0.f;
    *reinterpret_cast<uint4*>(out + q * C + 8 * g) = pack8(o);
  }
}

// Source planes of a batch: image b of r (or e) starts at ro.o[b], of U and V at uo.o[b].
struct Src {
  const double* r;
  const double* U;
  const double* V;
  int H, W, pitch;
};

// network input x = (r / rho, U, V, 0 ...) as 16 BF16 channels, zero on the padding
__global__ void k_net_in(Src s, Offs ro, Offs uo, const double* __restrict__ rho, int B, int Hn, int Wn,
                         bf16* __restrict__ xin, const int* skip) {
  if (skipped(skip)) return;
  const size_t n = (size_t)B * Hn * Wn;
  GRID_STRIDE(t, n) {
    const int j = (int)(t % Wn), i = (int)((t / Wn) % Hn), b = (int)(t / ((size_t)Wn * Hn));
    float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (i < s.H && j < s.W) {
      const double rb = rho[b];
      const double inv = rb > 0.0 ? 1.0 / rb : 0.0;
      const size_t o = (size_t)i * s.pitch + j;
      f[0] = (float)(s.r[ro.o[b] + o] * inv);
      f[1] = (float)s.U[uo.o[b] + o];
      f[2] = (float)s.V[uo.o[b] + o];
    }
    uint4* dst = reinterpret_cast<uint4*>(xin + t * 16);
    dst[0] = pack8(f);
    dst[1] = make_uint4(0, 0, 0, 0);
  }
}

// rho[b] = sqrt(mean over image b of x^2): block partials over a fixed element
// assignment, then one thread per image sums them in order.
constexpr int kStatBlocks = 64;
__global__ void __launch_bounds__(256) k_stats1(const double* __restrict__ x, Offs xo, int H, int W, int pitch,
                                                double* __restrict__ part, const int* skip) {
  if (skipped(skip)) return;
  const int b = blockIdx.y;
  const size_t n = (size_t)H * W;
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / W), j = (int)(e % W);
    const double v = x[xo.o[b] + (size_t)i * pitch + j];
    acc += v * v;
  }
  __shared__ double sh[8];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w];
    part[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}
__global__ void k_stats2(const double* __restrict__ part, int nb, int B, double count, double* out, const int* skip) {
  if (skipped(skip)) return;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int k = 0; k < nb; ++k) s += part[(size_t)b * nb + k];
  out[b] = sqrt(s / count);
}

// D^-1 of Eq. (Axb) at (i, j) from the weight planes (0 where D = 0)
__device__ __forceinline__ double dinv_at(const double* __restrict__ U, const double* __restrict__ V, int i, int j,
                                          size_t pitch) {
  const size_t o = (size_t)i * pitch + j;
  double d = U[o] + V[o];
  if (j > 0) d += U[o - 1];
  if (i > 0) d += V[o - pitch];
  return d > 0.0 ? 1.0 / d : 0.0;
}

// Direction loss of the training pairs (images of H x W, pitch W).  x = r / rho,
// s~ = D^-1 x + y (y the network output), e~ = e / rho:
//   L_b = 1 - (s~^T x)^2 / ((s~^T A s~)(e~^T x)),  dL_b/dy = c1 x + c2 A s~,
//   c1 = -2 a / (b g), c2 = 2 a^2 / (b^2 g),  a = s~^T x, b = s~^T A s~, g = e~^T x.
__global__ void k_dir_s(Src s, Offs ro, Offs uo, const double* __restrict__ rho, const float* __restrict__ y, int B,
                        double* __restrict__ sd) {
  const int H = s.H, W = s.W;
  const size_t n = (size_t)B * H * W;
  GRID_STRIDE(q, n) {
    const int j = (int)(q % W), i = (int)((q / W) % H), b = (int)(q / ((size_t)W * H));
    const double inv = rho[b] > 0.0 ? 1.0 / rho[b] : 0.0;
    const size_t o = (size_t)i * W + j;
    const double x = s.r[ro.o[b] + o] * inv;
    sd[q] = dinv_at(s.U + uo.o[b], s.V + uo.o[b], i, j, W) * x + (double)y[q];
  }
}

__global__ void __launch_bounds__(256) k_dir_stats(Src s, Offs ro, Offs uo, const double* __restrict__ e,
                                                   const double* __restrict__ rho, const double* __restrict__ sd,
                                                   double* __restrict__ asd, double* __restrict__ part) {
  const int b = blockIdx.y, H = s.H, W = s.W;
  const size_t n = (size_t)H * W;
  const double inv = rho[b] > 0.0 ? 1.0 / rho[b] : 0.0;
  const double* U = s.U + uo.o[b];
  const double* V = s.V + uo.o[b];
  const double* sb = sd + (size_t)b * n;
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / W), j = (int)(t % W);
    const double sc = sb[t];
    double d = U[t] + V[t];
    double as = 0.0;
    if (j + 1 < W) as -= U[t] * sb[t + 1];
    if (j > 0) {
      d += U[t - 1];
      as -= U[t - 1] * sb[t - 1];
    }
    if (i + 1 < H) as -= V[t] * sb[t + W];
    if (i > 0) {
      d += V[t - W];
      as -= V[t - W] * sb[t - W];
    }
    as += d * sc;
    asd[(size_t)b * n + t] = as;
    const double x = s.r[ro.o[b] + t] * inv;
    acc[0] += sc * x;
    acc[1] += sc * as;
    acc[2] += e[ro.o[b] + t] * inv * x;
  }
  __shared__ double sh[8][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double v = warp_sum(acc[k]);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += sh[w][threadIdx.x];
    part[((size_t)b * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = v;
  }
}

// per image: coefficients c1, c2 (scaled by 1/B) into coef[2b], coef[2b+1]; the batch loss
__global__ void k_dir_reduce(const double* __restrict__ part, int nb, int B, double* __restrict__ coef,
                             double* __restrict__ loss) {
  if (threadIdx.x != 0) return;
  double L = 0.0;
  for (int b = 0; b < B; ++b) {
    double a = 0.0, bb = 0.0, g = 0.0;
    for (int k = 0; k < nb; ++k) {
      a += part[((size_t)b * nb + k) * 3 + 0];
      bb += part[((size_t)b * nb + k) * 3 + 1];
      g += part[((size_t)b * nb + k) * 3 + 2];
    }
    const bool ok = bb > 0.0 && g > 0.0;
    coef[2 * b] = ok ? -2.0 * a / (bb * g) / B : 0.0;
    coef[2 * b + 1] = ok ? 2.0 * a * a / (bb * bb * g) / B : 0.0;
    L += ok ? 1.0 - a * a / (bb * g) : 1.0;
  }
  *loss = L / B;
}

__global__ void k_dir_grad(Src s, Offs ro, const double* __restrict__ rho, const double* __restrict__ asd,
                           const double* __restrict__ coef, int B, float* __restrict__ dy) {
  const int H = s.H, W = s.W;
  const size_t n = (size_t)B * H * W;
  GRID_STRIDE(q, n) {
    const size_t t = q % ((size_t)H * W);
    const int b = (int)(q / ((size_t)W * H));
    const double inv = rho[b] > 0.0 ? 1.0 / rho[b] : 0.0;
    const double x = s.r[ro.o[b] + t] * inv;
    dy[q] = (float)(coef[2 * b] * x + coef[2 * b + 1] * asd[q]);
  }
}

__device__ __forceinline__ float head_dot(const bf16* g, const float* hw, float hb, float (&f)[16]) {
  unpack8(reinterpret_cast<const uint4*>(g)[0], *reinterpret_cast<float(*)[8]>(&f[0]));
  unpack8(reinterpret_cast<const uint4*>(g)[1], *reinterpret_cast<float(*)[8]>(&f[8]));
  float y = hb;
#pragma unroll
  for (int c = 0; c < 16; ++c) y = fmaf(hw[c], f[c], y);
  return y;
}

// preconditioner output s = D^-1 r + rho * y (0 on masked pixels), FP64 plane with the given pitch
__global__ void k_head_apply(const bf16* __restrict__ g0, const float* __restrict__ hwp, const double* __restrict__ rho,
                             const double* __restrict__ r, const double* __restrict__ U, const double* __restrict__ V,
                             int H, int W, int Wn, const uint8_t* __restrict__ mask, int pitch, double* __restrict__ s,
                             const int* skip) {
  if (skipped(skip)) return;
  float hw[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) hw[c] = hwp[c];
  const float hb = hwp[16];
  const double rb = rho[0];
  const size_t n = (size_t)H * W;
  GRID_STRIDE(q, n) {
    const int j = (int)(q % W), i = (int)(q / W);
    float f[16];
    const float y = head_dot(g0 + ((size_t)i * Wn + j) * 16, hw, hb, f);
    const size_t o = (size_t)i * pitch + j;
    s[o] = (mask && mask[o]) ? 0.0 : dinv_at(U, V, i, j, pitch) * r[o] + rb * (double)y;
  }
}

// network output y (FP32, [B][Hn][Wn]) for the step-level forward entry point
__global__ void k_head_out(const bf16* __restrict__ g0, const float* __restrict__ hwp, size_t n, float* __restrict__ y) {
  float hw[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) hw[c] = hwp[c];
  const float hb = hwp[16];
  GRID_STRIDE(q, n) {
    float f[16];
    y[q] = head_dot(g0 + q * 16, hw, hb, f);
  }
}

// head backward: d = dL/dy; dg0 = d * w_h * (g0 > 0); block partials of sum d g0[c] (16), sum d
constexpr int kHeadBlocks = 512;
__global__ void __launch_bounds__(256) k_head_train(const bf16* __restrict__ g0, const float* __restrict__ hwp,
                                                    const float* __restrict__ dyp, size_t n, bf16* __restrict__ dg0,
                                                    double* __restrict__ part) {
  float hw[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) hw[c] = hwp[c];
  double acc[17];
#pragma unroll
  for (int k = 0; k < 17; ++k) acc[k] = 0.0;
  GRID_STRIDE(q, n) {
    float f[16];
    head_dot(g0 + q * 16, hw, 0.f, f);
    const double d = (double)dyp[q];
    float o0[8], o1[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      o0[c] = f[c] > 0.f ? (float)(d * hw[c]) : 0.f;
      o1[c] = f[8 + c] > 0.f ? (float)(d * hw[8 + c]) : 0.f;
    }
    uint4* dst = reinterpret_cast<uint4*>(dg0 + q * 16);
    dst[0] = pack8(o0);
    dst[1] = pack8(o1);
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] += d * (double)f[c];
    acc[16] += d;
  }
  __shared__ double sh[8][17];
#pragma unroll
  for (int k = 0; k < 17; ++k) {
    const double v = warp_sum(acc[k]);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 17) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w][threadIdx.x];
    part[(size_t)blockIdx.x * 17 + threadIdx.x] = s;
  }
}
__global__ void k_head_reduce(const double* __restrict__ part, int nb, float* __restrict__ ghead) {
  const int k = threadIdx.x;
  if (k >= 17) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(size_t)b * 17 + k];
  ghead[k] = (float)s;
}

// ------------------------------------------------------------------ weight gradient
// dW[o][c][t] = sum_p dy[p][o] x[p + off(t)][c] and db[o] = sum_p dy[p][o] as one GEMM
// on the tensor cores with the pixels as the reduction dimension:
//   D[m][o] = sum_p A[m][p] B[o][p],  A[c 9 + t][p] = x[p + off(t)][c] (0 outside the
//   image), A[9 C][p] = 1 (the bias row), B[o][p] = dy[p][o].
// The m rows come in 128-row tiles; a CTA owns a group of consecutive tiles (their
// accumulators side by side in tensor memory, G x O <= 512 columns) and a contiguous
// range of pixel chunks (split K).  A chunk is a bw x bh block of 64 pixels of one
// image (bw the largest power of two dividing W, at most 64); chunks are numbered down
// each bw-wide column strip, so a CTA's consecutive chunks share all but bh of the
// bh + 2 input rows that their 3 x 3 taps read.  Those rows are kept in a shared-memory
// ring (only the new rows are loaded, as 16-byte pieces of 8 channels, zero outside the
// image) together with the chunk's dy.  From them the 128 threads build, per chunk, the
// B tile once and each tile's A rows (one row per thread) in the canonical K-major
// layout with the 128-byte swizzle (8-row atoms of 1024 bytes; the 16-byte piece j of
// row r stored at piece j ^ (r mod 8)), and one thread issues four K = 16 MMAs per tile
// into its FP32 accumulator; the A tiles alternate between two buffers, so a tile's MMAs
// run while the next tile is built.  Partials go to part[split][m][o] and a second kernel
// sums the splits in order, so the result does not depend on scheduling.
constexpr int kWgA = 128 * 128;                  // one A tile: 128 rows x 64 pixels x 2 bytes
constexpr int kWgHaloBytes = 48 * 1024;          // input-row ring: (2 bh + 2) rows x (bw + 2) pixels x channels
constexpr int kWgSmem = 2 * kWgA + 128 * 128 + kWgHaloBytes + 2 * 64 * 128 * 2 + 1024 + 256;  // the largest layout
constexpr size_t kPartFloats = (size_t)kPartRows * kPartCols;

struct WgArgs {
  const bf16* dy;   // [P][O]
  const bf16* x;    // [P][Cx], channels [0, C) used
  int O, Cx, C, B, H, W, bw, lbw, bh;
  int mtiles, gtiles;   // 128-row tiles of m = 9 C + 1 rows, tiles per CTA group
  int chunks;       // pixel chunks of the whole batch
  int per_split;    // chunks per CTA
  int tcols;        // tensor-memory columns allocated (>= gtiles O, power of two, >= 32)
  int off_ring, off_dy, off_bar;  // shared-memory layout (bytes from the 1024-aligned base)
  float* part;      // [split][mtiles * 128][O]
  int* err;
};

__device__ __forceinline__ uint32_t sw128_off(int row, int piece) {
  return (uint32_t)(row * 128 + ((piece ^ (row & 7)) << 4));
}

// 16-byte asynchronous copy into shared memory, zero-filled when !valid (nothing is read then)
__device__ __forceinline__ void cpa16(void* sdst, const void* gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(sdst)), "l"(gsrc),
               "r"(valid ? 16 : 0)
               : "memory");
}

// NP: 8-channel pieces per ring pixel (the largest of the layer's groups), so the ring's
// channel stride is a compile-time constant.  256 threads: each A row is built by two
// threads (four 16-byte pieces each).
constexpr int kWgThreads = 256;
template <int NP>
__global__ void __launch_bounds__(kWgThreads) k_wgrad_tc(WgArgs a) {
  constexpr int HS = NP * 8;                                  // ring channels per pixel
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* sbt = base + 2 * kWgA;                       // the B tile (O rows)
  unsigned char* ring = base + a.off_ring;                    // [slot][pixel][HS channels]
  bf16* sdy = reinterpret_cast<bf16*>(base + a.off_dy);       // 2 x [q][O]
  uint64_t* a_done = reinterpret_cast<uint64_t*>(base + a.off_bar);
  uint64_t* b_done = a_done + 2;
  uint64_t* fin = b_done + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ int s_rowbase[10];                               // ring offset (pixels) of window row w
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = blockIdx.x, split = blockIdx.y;
  const int t0 = grp * a.gtiles, G = min(a.gtiles, a.mtiles - t0);
  const int k0 = split * a.per_split, k1 = min(a.chunks, k0 + a.per_split);
  const uint32_t idesc = idesc_bf16(128, a.O);
  if (tid == 0) {
    mbar_init(a_done, 1);
    mbar_init(a_done + 1, 1);
    mbar_init(b_done, 1);
    mbar_init(fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  // channels of the group's rows: [cb0, cb0 + 8 np) (whole pieces inside the pixel), np <= NP
  const int c_first = min((t0 * 128) / 9, a.C - 1), c_last = min(a.C - 1, ((t0 + G) * 128 - 1) / 9);
  const int cb0 = c_first & ~7;
  const int np = (c_last - cb0) / 8 + 1;
  const int hbw = a.bw + 2, nslot = a.bh + 2, nring = 2 * a.bh + 2;  // window rows; ring slots
  const int hw = a.H * a.W, nrb = a.H / a.bh, nstrip = a.W / a.bw;
  const unsigned short one = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
  const int r128 = tid & 127, half = tid >> 7;                // the A row slot and piece half of this thread
  // this thread's row of a tile, taken in tap-major order (the lanes of a warp then read
  // neighbouring channels of one tap, not one channel at nine taps)
  auto my_row = [&](int M0, int& t, int& c) {
    int rem = r128;
    t = 8;
    c = 0;
    for (int tt = 0; tt < 9; ++tt) {
      const int cmin = (M0 - tt + 8) / 9, cmax = (M0 + 127 - tt) / 9;  // M0 - tt >= -8
      const int n = cmax - cmin + 1;
      if (rem < n) { t = tt; c = cmin + rem; return; }
      rem -= n;
    }
  };
  // asynchronous copies of rows a in [a0, a1) of the chunk's column strip (image b, columns
  // x0 - 1 .. x0 + bw) into their ring slots (a + 1) mod nring, zero outside the image
  auto load_rows = [&](int b, int x0, int a0, int a1) {
    const int n = (a1 - a0) * hbw * np;
    for (int e = tid; e < n; e += kWgThreads) {
      const int pc = e % np, rest = e / np;
      const int col = rest % hbw, py = a0 + rest / hbw, px = x0 - 1 + col;
      const bool in = py >= 0 && py < a.H && px >= 0 && px < a.W;
      const bf16* src = in ? a.x + ((size_t)b * hw + (size_t)py * a.W + px) * a.Cx + cb0 + 8 * pc : a.x;
      cpa16(ring + ((size_t)(((py + 1) % nring) * hbw + col) * NP + pc) * 16, src, in);
    }
  };
  auto load_dy = [&](int b, int y0, int x0, bf16* dst) {
    const int opc = a.O / 8;
    for (int e = tid; e < 64 * opc; e += kWgThreads) {
      const int q = e / opc, pc = e - q * opc;
      const int py = y0 + (q >> a.lbw), px = x0 + (q & (a.bw - 1));
      cpa16(dst + q * a.O + 8 * pc, a.dy + ((size_t)b * hw + (size_t)py * a.W + px) * a.O + 8 * pc, true);
    }
  };
  auto chunk_at = [&](int k, int& b, int& y0, int& x0) {
    const int ry = k % nrb, sx = (k / nrb) % nstrip;
    b = k / (nrb * nstrip);
    y0 = ry * a.bh;
    x0 = sx * a.bw;
  };
  bool ok = true;
  int u = 0;  // A-tile builds so far (buffer u & 1)
  bool have_rows = false;  // the current chunk's new rows were prefetched by the previous iteration
  for (int k = k0; k < k1 && ok; ++k) {
    const int i = k - k0;
    int b, y0, x0;
    chunk_at(k, b, y0, x0);
    bf16* dyc = sdy + (i & 1) * 64 * a.O;
    if (!have_rows) {  // the first chunk of the CTA, or one that starts another strip: all its rows
      load_rows(b, x0, y0 - 1, y0 + a.bh + 1);
      if (i == 0) load_dy(b, y0, x0, dyc);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // prefetch the next chunk: its dy, and its bh new rows when it follows in the same strip
    have_rows = false;
    if (k + 1 < k1) {
      int b2, y2, x2;
      chunk_at(k + 1, b2, y2, x2);
      load_dy(b2, y2, x2, sdy + ((i + 1) & 1) * 64 * a.O);
      if (b2 == b && x2 == x0 && y2 == y0 + a.bh) {
        load_rows(b, x0, y2 + 1, y2 + a.bh + 1);
        have_rows = true;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // this chunk's copies (not the prefetch)
    if (tid < nslot) s_rowbase[tid] = ((y0 + tid) % nring) * hbw;  // window row w = abs row y0 - 1 + w
    // the previous chunk's MMAs must have read the B tile
    if (i > 0) ok = ok && mbar_wait(b_done, (i - 1) & 1, a.err);
    if (!__syncthreads_and(ok)) { ok = false; break; }
    if (tid < 2 * a.O) {
      const int o = tid % a.O, h = tid / a.O;
      const unsigned short* src = reinterpret_cast<const unsigned short*>(dyc) + o;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = 4 * h + jj;
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          w[e] = (uint32_t)src[(8 * j + 2 * e) * a.O] | ((uint32_t)src[(8 * j + 2 * e + 1) * a.O] << 16);
        *reinterpret_cast<uint4*>(sbt + sw128_off(o, j)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    for (int g = 0; g < G; ++g, ++u) {
      unsigned char* sa = base + (u & 1) * kWgA;
      if (u >= 2) ok = ok && mbar_wait(a_done + (u & 1), ((u - 2) >> 1) & 1, a.err);
      const int M0 = (t0 + g) * 128;
      int t, c;
      my_row(M0, t, c);
      const int m = 9 * c + t, row = m - M0;
      const bool xrow = m < 9 * a.C, brow = m == 9 * a.C;
      const int ty = t / 3, tx = t - 3 * ty;
      const unsigned short* hr = reinterpret_cast<const unsigned short*>(ring) + (c - cb0);
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = 4 * half + jj;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (xrow) {
          // the piece's 8 pixels lie in one row of the block (bw >= 8)
          const int q0 = 8 * j;
          const unsigned short* src = hr + (s_rowbase[(q0 >> a.lbw) + ty] + (q0 & (a.bw - 1)) + tx) * HS;
#pragma unroll
          for (int e = 0; e < 4; ++e) w[e] = (uint32_t)src[2 * e * HS] | ((uint32_t)src[(2 * e + 1) * HS] << 16);
        } else if (brow) {
          w[0] = w[1] = w[2] = w[3] = (uint32_t)one | ((uint32_t)one << 16);
        }
        *reinterpret_cast<uint4*>(sa + sw128_off(row, j)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
      // the generic-proxy stores must be visible to the tensor cores' reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (!__syncthreads_and(ok)) { ok = false; break; }
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t da = sw128_desc(sa), db = sw128_desc(sbt);
        const uint32_t acc_col = tmem + (uint32_t)(g * a.O);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(acc_col, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (i | kk) != 0);
        mma_commit(a_done + (u & 1));
        if (g == G - 1) mma_commit(b_done);
      }
    }
    // the prefetched rows and dy are complete, and every thread is done with this chunk's
    // window before the next iteration's prefetch overwrites its oldest rows
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (tid == 0) mma_commit(fin);
  __syncwarp();
  const bool ready = __all_sync(0xffffffffu, ok && mbar_wait(fin, 0, a.err)) && k1 > k0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warps w and w + 4 read the lane quarter w & 3 of every accumulator, each
  // half of its 16-column chunks
  const int quarter = warp & 3, chalf = warp >> 2, nq = a.O >> 4;
  for (int g = 0; g < G; ++g) {
    float* dst = a.part + (((size_t)split * a.mtiles + t0 + g) * 128 + quarter * 32 + lane) * a.O;
    for (int cq = chalf; cq < nq; cq += 2) {
      if (ready) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * a.O + cq * 16), v);
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4*>(dst + cq * 16 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      } else {
        for (int q = 0; q < 16; ++q) dst[cq * 16 + q] = 0.f;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tcols));
}

// canonical gradient of one layer: W [O][C][3][3] at gw, bias [O] at gb; sums the
// splits of part[split][m][o] (m = c 9 + t, the bias row at m = 9 C) in order.  Thread e
// takes (m, o) = (e / O, e mod O), so a warp reads consecutive o of one row.
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nsplit, int mtiles, int O, int C,
                               float* __restrict__ gw, float* __restrict__ gb) {
  const int n = (9 * C + 1) * O;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int m = e / O, o = e - m * O;
    double s = 0.0;
    for (int g = 0; g < nsplit; ++g) s += part[((size_t)g * mtiles * 128 + m) * O + o];
    if (m < 9 * C) gw[(size_t)o * 9 * C + m] = (float)s;  // W[o][c][t] at o 9 C + c 9 + t
    else gb[o] = (float)s;
  }
}

// once per device, before any capture
static cudaError_t conv_init() {
  const cudaError_t e = cudaFuncSetAttribute(k_conv3x3, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_smem(256));
  if (e != cudaSuccess) return e;
  const void* fns[] = {(const void*)k_wgrad_tc<1>, (const void*)k_wgrad_tc<2>, (const void*)k_wgrad_tc<3>,
                       (const void*)k_wgrad_tc<4>, (const void*)k_wgrad_tc<5>, (const void*)k_wgrad_tc<6>,
                       (const void*)k_wgrad_tc<7>, (const void*)k_wgrad_tc<8>, (const void*)k_wgrad_tc<9>,
                       (const void*)k_wgrad_tc<10>, (const void*)k_wgrad_tc<11>, (const void*)k_wgrad_tc<12>};
  for (const void* f : fns) {
    const cudaError_t e2 = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
    if (e2 != cudaSuccess) return e2;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ parameters
// wf[o][t][c] = W[o][c][t] (c < Cin, zero up to CinPad); wb[c][t][o] = W[o][c][8 - t]
__global__ void k_repack(const float* __restrict__ theta, long long woff, int O, int C, int CP, bf16* __restrict__ wf,
                         bf16* __restrict__ wb) {
  const int n = O * 9 * CP;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int c = e % CP, t = (e / CP) % 9, o = e / (9 * CP);
    wf[e] = __float2bfloat16_rn(c < C ? theta[woff + ((size_t)o * C + c) * 9 + t] : 0.f);
    if (wb && c < C) wb[((size_t)c * 9 + t) * O + o] = __float2bfloat16_rn(theta[woff + ((size_t)o * C + c) * 9 + (8 - t)]);
  }
}

__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    theta[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace unet

// ------------------------------------------------------------------ the network object
using namespace unet;

struct Unet {
  int device = 0;
  Offsets off{};
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  long long step = 0;
  bf16* wf[kNL] = {};
  bf16* wb[kNL] = {};
  void* wmem = nullptr;
  int* err = nullptr;
  double* red = nullptr;      // per-image statistics and reduction partials
  float* part = nullptr;      // weight-gradient partials
  // activation workspace for (B, Hn, Wn)
  int wsB = 0, wsH = 0, wsW = 0;
  long long ws_gen = 0;       // incremented whenever the workspace moves
  void* ws = nullptr;
  bf16 *xin = nullptr, *cat0 = nullptr, *p0 = nullptr, *cat1 = nullptr, *p1 = nullptr, *cat2 = nullptr,
       *p2 = nullptr, *g0 = nullptr;
  bf16 *dg0 = nullptr, *dcat0 = nullptr, *dg1 = nullptr, *dcat1 = nullptr, *dg2 = nullptr, *dcat2 = nullptr,
       *da3 = nullptr, *dp2 = nullptr, *da2 = nullptr, *dp1 = nullptr, *da1 = nullptr, *dp0 = nullptr,
       *da0 = nullptr;
  float *y = nullptr, *t = nullptr;  // network output; dL/dy
  double *sd = nullptr, *asd = nullptr;  // training: s~ and A s~
};

// reduction scratch layout (doubles)
constexpr int kRedRho = 0, kRedLoss = 64, kRedCoef = 128, kRedPart = 256;
constexpr size_t kRedHead = kRedPart + (size_t)kMaxBatch * kStatBlocks;       // head partials
constexpr size_t kRedDir = kRedHead + (size_t)kHeadBlocks * 17;               // direction-loss partials
constexpr size_t kRedDoubles = kRedDir + (size_t)kMaxBatch * kStatBlocks * 3;

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Allocates the activation workspace for batches of B images of Hn x Wn (multiples of 128).
int unet_prepare(Unet& u, int B, int Hn, int Wn) {
  if (u.ws && B <= u.wsB && Hn == u.wsH && Wn == u.wsW) return 0;
  if (u.ws) cudaFree(u.ws);
  u.ws = nullptr;
  const size_t P0 = (size_t)B * Hn * Wn, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  struct Item {
    bf16** p;
    size_t elems;
  } items[] = {{&u.xin, P0 * 16},  {&u.cat0, P0 * 48}, {&u.p0, P1 * 16},   {&u.cat1, P1 * 96},
               {&u.p1, P2 * 32},   {&u.cat2, P2 * 192}, {&u.p2, P3 * 64},  {&u.g0, P0 * 16},
               {&u.dg0, P0 * 16},  {&u.dcat0, P0 * 48}, {&u.dg1, P1 * 32}, {&u.dcat1, P1 * 96},
               {&u.dg2, P2 * 64},  {&u.dcat2, P2 * 192}, {&u.da3, P3 * 128}, {&u.dp2, P3 * 64},
               {&u.da2, P2 * 64},  {&u.dp1, P2 * 32},  {&u.da1, P1 * 32}, {&u.dp0, P1 * 16},
               {&u.da0, P0 * 16}};
  size_t bytes = 0;
  for (const Item& it : items) bytes += align256(it.elems * 2);
  bytes += 2 * align256(P0 * 4) + 2 * align256(P0 * 8);
  char* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return -5;
  if (cudaMemset(p, 0, bytes) != cudaSuccess) {
    cudaFree(p);
    return -2;
  }
  u.ws = p;
  for (const Item& it : items) {
    *it.p = reinterpret_cast<bf16*>(p);
    p += align256(it.elems * 2);
  }
  u.y = reinterpret_cast<float*>(p);
  p += align256(P0 * 4);
  u.t = reinterpret_cast<float*>(p);
  p += align256(P0 * 4);
  u.sd = reinterpret_cast<double*>(p);
  p += align256(P0 * 8);
  u.asd = reinterpret_cast<double*>(p);
  u.wsB = B;
  u.wsH = Hn;
  u.wsW = Wn;
  u.ws_gen += 1;
  return 0;
}

long long unet_ws_gen(const Unet& u) { return u.ws_gen; }

static cudaError_t repack(Unet& u, cudaStream_t st) {
  for (int l = 0; l < kNL; ++l) {
    const int n = kCout[l] * 9 * kCinPad[l];
    k_repack<<<(n + 255) / 256, 256, 0, st>>>(u.theta, u.off.w[l], kCout[l], kCin[l], kCinPad[l], u.wf[l],
                                             l == E0 ? nullptr : u.wb[l]);
  }
  return cudaGetLastError();
}

static int eblocks(size_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

// Forward pass on the prepared workspace: xin -> ... -> g0 (d0's activations).
static cudaError_t forward(Unet& u, int B, int Hn, int Wn, const int* skip, cudaStream_t st) {
  const int H1 = Hn / 2, W1 = Wn / 2, H2 = Hn / 4, W2 = Wn / 4, H3 = Hn / 8, W3 = Wn / 8;
  const float* th = u.theta;
  cudaError_t e;
#define CK(x) \
  if ((e = (x)) != cudaSuccess) return e
  CK(conv3x3(u.xin, B, Hn, Wn, 16, u.wf[E0], 16, th + u.off.b[E0], 1, u.cat0, 48, 0, 0, skip, u.err, st));
  k_pool2<<<eblocks((size_t)B * H1 * W1 * 2), 256, 0, st>>>(u.cat0, 48, 16, B, Hn, Wn, u.p0, skip);
  CK(conv3x3(u.p0, B, H1, W1, 16, u.wf[E1], 32, th + u.off.b[E1], 1, u.cat1, 96, 0, 0, skip, u.err, st));
  k_pool2<<<eblocks((size_t)B * H2 * W2 * 4), 256, 0, st>>>(u.cat1, 96, 32, B, H1, W1, u.p1, skip);
  CK(conv3x3(u.p1, B, H2, W2, 32, u.wf[E2], 64, th + u.off.b[E2], 1, u.cat2, 192, 0, 0, skip, u.err, st));
  k_pool2<<<eblocks((size_t)B * H3 * W3 * 8), 256, 0, st>>>(u.cat2, 192, 64, B, H2, W2, u.p2, skip);
  CK(conv3x3(u.p2, B, H3, W3, 64, u.wf[B3], 128, th + u.off.b[B3], 1, u.cat2, 192, 64, 1, skip, u.err, st));
  CK(conv3x3(u.cat2, B, H2, W2, 192, u.wf[D2], 64, th + u.off.b[D2], 1, u.cat1, 96, 32, 1, skip, u.err, st));
  CK(conv3x3(u.cat1, B, H1, W1, 96, u.wf[D1], 32, th + u.off.b[D1], 1, u.cat0, 48, 16, 1, skip, u.err, st));
  CK(conv3x3(u.cat0, B, Hn, Wn, 48, u.wf[D0], 16, th + u.off.b[D0], 1, u.g0, 16, 0, 0, skip, u.err, st));
  return cudaGetLastError();
}

static cudaError_t wgrad(Unet& u, int l, const bf16* dy, const bf16* x, int Cx, int B, int H, int W,
                         cudaStream_t st) {
  WgArgs a{};
  a.dy = dy;
  a.x = x;
  a.O = kCout[l];
  a.Cx = Cx;
  a.C = kCin[l];
  a.B = B;
  a.H = H;
  a.W = W;
  a.bw = W & -W;
  if (a.bw > 64) a.bw = 64;
  a.lbw = 0;
  while ((1 << a.lbw) < a.bw) ++a.lbw;
  a.bh = 64 / a.bw;
  if (a.bw < 8 || a.bh > H || H % a.bh || a.O % 16 || a.O > 128 || Cx % 8) return cudaErrorInvalidValue;
  a.mtiles = (9 * a.C + 1 + 127) / 128;
  // tiles per group: their accumulators fit tensor memory, and the channels they read
  // fit the input-row ring (the tile rows of one group span about 14 G + 1 channels)
  const int ring_px = (2 * a.bh + 2) * (a.bw + 2);  // ring slots x (bw + 2) pixels
  a.gtiles = 512 / a.O;
  auto pieces = [](int g) { return ((g * 128) / 9 + 1 + 7 + 7) / 8; };  // 8-channel pieces a group may read
  while (a.gtiles > 1 && (pieces(a.gtiles) * 16 * ring_px > kWgHaloBytes || pieces(a.gtiles) > 12)) --a.gtiles;
  if (a.gtiles > a.mtiles) a.gtiles = a.mtiles;
  const int ngroups = (a.mtiles + a.gtiles - 1) / a.gtiles;
  // every group's channel pieces inside the pixel and its rows inside the ring (as the kernel forms them)
  for (int grp = 0; grp < ngroups; ++grp) {
    const int t0 = grp * a.gtiles, G = a.gtiles < a.mtiles - t0 ? a.gtiles : a.mtiles - t0;
    const int cf = ((t0 * 128) / 9 < a.C - 1) ? (t0 * 128) / 9 : a.C - 1;
    const int cl = (((t0 + G) * 128 - 1) / 9 < a.C - 1) ? ((t0 + G) * 128 - 1) / 9 : a.C - 1;
    const int np = (cl - (cf & ~7)) / 8 + 1;
    if ((cf & ~7) + 8 * np > Cx || (long long)ring_px * np * 16 > kWgHaloBytes) return cudaErrorInvalidValue;
  }
  a.chunks = B * (H / a.bh) * (W / a.bw);
  // about four CTAs per SM in all, within the partial buffer
  long long nsplit = (4LL * 152 + ngroups - 1) / ngroups;
  const long long cap = (long long)(kPartFloats / ((size_t)a.mtiles * 128 * a.O));
  if (nsplit > cap) nsplit = cap;
  if (nsplit > a.chunks) nsplit = a.chunks;
  if (nsplit < 1) nsplit = 1;
  a.per_split = (int)((a.chunks + nsplit - 1) / nsplit);
  nsplit = (a.chunks + a.per_split - 1) / a.per_split;
  a.tcols = 32;
  while (a.tcols < a.gtiles * a.O) a.tcols <<= 1;
  a.part = u.part;
  a.err = u.err;
  // shared memory: two A tiles, the B tile (O rows), the ring (the largest group's pieces),
  // the chunk's dy, the barriers; sized per layer so that several CTAs share an SM
  int np_max = 1;
  for (int grp = 0; grp < ngroups; ++grp) {
    const int t0 = grp * a.gtiles, G = a.gtiles < a.mtiles - t0 ? a.gtiles : a.mtiles - t0;
    const int cf = ((t0 * 128) / 9 < a.C - 1) ? (t0 * 128) / 9 : a.C - 1;
    const int cl = (((t0 + G) * 128 - 1) / 9 < a.C - 1) ? ((t0 + G) * 128 - 1) / 9 : a.C - 1;
    const int np = (cl - (cf & ~7)) / 8 + 1;
    if (np > np_max) np_max = np;
  }
  a.off_ring = 2 * kWgA + a.O * 128;
  a.off_dy = a.off_ring + ((ring_px * np_max * 16 + 127) & ~127);
  a.off_bar = a.off_dy + 2 * ((64 * a.O * 2 + 127) & ~127);
  const int smem = a.off_bar + 64 + 1024;
  if (smem > kWgSmem) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)ngroups, (unsigned)nsplit);
  switch (np_max) {
#define WG_CASE(N) \
  case N: k_wgrad_tc<N><<<grid, kWgThreads, smem, st>>>(a); break;
    WG_CASE(1) WG_CASE(2) WG_CASE(3) WG_CASE(4) WG_CASE(5) WG_CASE(6) WG_CASE(7) WG_CASE(8) WG_CASE(9)
    WG_CASE(10) WG_CASE(11) WG_CASE(12)
#undef WG_CASE
    default: return cudaErrorInvalidValue;
  }
  const int n = (9 * a.C + 1) * a.O;
  k_wgrad_reduce<<<(n + 255) / 256, 256, 0, st>>>(u.part, (int)nsplit, a.mtiles, a.O, a.C, u.grad + u.off.w[l],
                                                  u.grad + u.off.b[l]);
  return cudaGetLastError();
}

// Backward pass: from the loss on y against t to u.grad (canonical layout) and the loss.
static cudaError_t backward(Unet& u, int B, int Hn, int Wn, cudaStream_t st) {
  const int H1 = Hn / 2, W1 = Wn / 2, H2 = Hn / 4, W2 = Wn / 4, H3 = Hn / 8, W3 = Wn / 8;
  const size_t n = (size_t)B * Hn * Wn;
  cudaError_t e;
  double* part = u.red + kRedHead;
  k_head_train<<<kHeadBlocks, 256, 0, st>>>(u.g0, u.theta + u.off.hw, u.t, n, u.dg0, part);
  k_head_reduce<<<1, 32, 0, st>>>(part, kHeadBlocks, u.grad + u.off.hw);
  // d0
  CK(wgrad(u, D0, u.dg0, u.cat0, 48, B, Hn, Wn, st));
  CK(conv3x3(u.dg0, B, Hn, Wn, 16, u.wb[D0], 48, nullptr, 0, u.dcat0, 48, 0, 0, nullptr, u.err, st));
  k_upsum_gate<<<eblocks((size_t)B * H1 * W1 * 4), 256, 0, st>>>(u.dcat0, u.cat0, 48, 16, 32, B, H1, W1, u.dg1);
  // d1
  CK(wgrad(u, D1, u.dg1, u.cat1, 96, B, H1, W1, st));
  CK(conv3x3(u.dg1, B, H1, W1, 32, u.wb[D1], 96, nullptr, 0, u.dcat1, 96, 0, 0, nullptr, u.err, st));
  k_upsum_gate<<<eblocks((size_t)B * H2 * W2 * 8), 256, 0, st>>>(u.dcat1, u.cat1, 96, 32, 64, B, H2, W2, u.dg2);
  // d2
  CK(wgrad(u, D2, u.dg2, u.cat2, 192, B, H2, W2, st));
  CK(conv3x3(u.dg2, B, H2, W2, 64, u.wb[D2], 192, nullptr, 0, u.dcat2, 192, 0, 0, nullptr, u.err, st));
  k_upsum_gate<<<eblocks((size_t)B * H3 * W3 * 16), 256, 0, st>>>(u.dcat2, u.cat2, 192, 64, 128, B, H3, W3, u.da3);
  // b3
  CK(wgrad(u, B3, u.da3, u.p2, 64, B, H3, W3, st));
  CK(conv3x3(u.da3, B, H3, W3, 128, u.wb[B3], 64, nullptr, 0, u.dp2, 64, 0, 0, nullptr, u.err, st));
  k_merge_gate<<<eblocks((size_t)B * H2 * W2 * 8), 256, 0, st>>>(u.dcat2, u.cat2, 192, 64, u.dp2, B, H2, W2, u.da2);
  // e2
  CK(wgrad(u, E2, u.da2, u.p1, 32, B, H2, W2, st));
  CK(conv3x3(u.da2, B, H2, W2, 64, u.wb[E2], 32, nullptr, 0, u.dp1, 32, 0, 0, nullptr, u.err, st));
  k_merge_gate<<<eblocks((size_t)B * H1 * W1 * 4), 256, 0, st>>>(u.dcat1, u.cat1, 96, 32, u.dp1, B, H1, W1, u.da1);
  // e1
  CK(wgrad(u, E1, u.da1, u.p0, 16, B, H1, W1, st));
  CK(conv3x3(u.da1, B, H1, W1, 32, u.wb[E1], 16, nullptr, 0, u.dp0, 16, 0, 0, nullptr, u.err, st));
  k_merge_gate<<<eblocks((size_t)B * Hn * Wn * 2), 256, 0, st>>>(u.dcat0, u.cat0, 48, 16, u.dp0, B, Hn, Wn, u.da0);
  // e0 (no input gradient)
  CK(wgrad(u, E0, u.da0, u.xin, 16, B, Hn, Wn, st));
#undef CK
  return cudaGetLastError();
}

// rho of B images into out[b]
static void rms(Unet& u, const double* x, const Offs& xo, int B, int H, int W, int pitch, double* out,
                const int* skip, cudaStream_t st) {
  double* part = u.red + kRedPart;
  k_stats1<<<dim3(kStatBlocks, B), 256, 0, st>>>(x, xo, H, W, pitch, part, skip);
  k_stats2<<<1, 64, 0, st>>>(part, kStatBlocks, B, (double)H * W, out, skip);
}

// s = D^-1 r + rho N(r / rho, U, V) on one map (planes with the given pitch), 0 on masked pixels.
cudaError_t unet_apply_plane(Unet& u, const double* r, const double* U, const double* V, const uint8_t* mask, int H,
                             int W, int pitch, double* s, const int* skip, cudaStream_t st) {
  const int Hn = (H + 127) / 128 * 128, Wn = (W + 127) / 128 * 128;
  if (!u.ws || u.wsH != Hn || u.wsW != Wn || u.wsB < 1) return cudaErrorInvalidValue;
  Offs z{};
  rms(u, r, z, 1, H, W, pitch, u.red + kRedRho, skip, st);
  Src src{r, U, V, H, W, pitch};
  k_net_in<<<eblocks((size_t)Hn * Wn), 256, 0, st>>>(src, z, z, u.red + kRedRho, 1, Hn, Wn, u.xin, skip);
  const cudaError_t e = forward(u, 1, Hn, Wn, skip, st);
  if (e != cudaSuccess) return e;
  k_head_apply<<<eblocks((size_t)H * W), 256, 0, st>>>(u.g0, u.theta + u.off.hw, u.red + kRedRho, r, U, V, H, W,
                                                     Wn, mask, pitch, s, skip);
  return cudaGetLastError();
}

int unet_error(Unet& u) {
  int e = 0;
  cudaMemcpy(&e, u.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) cudaMemset(u.err, 0, sizeof(int));
  return e;
}

}  // namespace ulp

// ------------------------------------------------------------------ C ABI
using namespace ulp;

struct ulp_unet_s {
  Unet u;
};

static int unet_fail(int code, const char* msg) { return set_error(code, msg); }

ulp::Unet* ulp_unet_impl(ulp_unet net) { return &net->u; }

#define UCU(x)                                                                        \
  do {                                                                                \
    const cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                          \
      char b_[256];                                                                   \
      std::snprintf(b_, sizeof(b_), "%s: %s", #x, cudaGetErrorString(e_));            \
      return unet_fail(ULP_ERR_CUDA, b_);                                             \
    }                                                                                 \
  } while (0)

extern "C" int ulp_unet_param_count(void) { return (int)offsets().n; }

static unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

extern "C" int ulp_unet_create(unsigned long long seed, ulp_unet* out) {
  if (!out) return unet_fail(ULP_ERR_INVALID, "ulp_unet_create: null out");
  *out = nullptr;
  ulp_unet h = new ulp_unet_s();
  Unet& u = h->u;
  u.off = offsets();
  const size_t n = (size_t)u.off.n;
  size_t wbytes = 0;
  for (int l = 0; l < kNL; ++l) wbytes += 2 * align256((size_t)kCout[l] * 9 * kCinPad[l] * 2);
  const size_t bytes = 4 * align256(n * 4) + wbytes + 256 + align256(kRedDoubles * 8) +
                       align256((size_t)kPartRows * kPartCols * 4);
  char* p = nullptr;
  if (cudaGetDevice(&u.device) != cudaSuccess || cudaMalloc(&p, bytes) != cudaSuccess) {
    delete h;
    return unet_fail(ULP_ERR_NOMEM, "ulp_unet_create: device allocation failed");
  }
  cudaMemset(p, 0, bytes);
  u.wmem = p;
  u.theta = reinterpret_cast<float*>(p);
  p += align256(n * 4);
  u.grad = reinterpret_cast<float*>(p);
  p += align256(n * 4);
  u.m = reinterpret_cast<float*>(p);
  p += align256(n * 4);
  u.v = reinterpret_cast<float*>(p);
  p += align256(n * 4);
  for (int l = 0; l < kNL; ++l) {
    const size_t b = align256((size_t)kCout[l] * 9 * kCinPad[l] * 2);
    u.wf[l] = reinterpret_cast<bf16*>(p);
    p += b;
    u.wb[l] = reinterpret_cast<bf16*>(p);
    p += b;
  }
  u.err = reinterpret_cast<int*>(p);
  p += 256;
  u.red = reinterpret_cast<double*>(p);
  p += align256(kRedDoubles * 8);
  u.part = reinterpret_cast<float*>(p);
  // He-uniform initial weights, zero biases, small head
  std::vector<float> th(n, 0.f);
  unsigned long long k = 0;
  auto uni = [&](float a) {
    const unsigned long long z = splitmix64(seed ^ (0xA5A5A5A5ull + k++));
    return a * (2.f * (float)((z >> 11) * (1.0 / 9007199254740992.0)) - 1.f);
  };
  for (int l = 0; l < kNL; ++l) {
    const float a = std::sqrt(6.f / (9.f * kCin[l]));
    for (long long i = 0; i < (long long)kCout[l] * kCin[l] * 9; ++i) th[u.off.w[l] + i] = uni(a);
  }
  for (int c = 0; c < 16; ++c) th[u.off.hw + c] = uni(0.25f);
  if (conv_init() != cudaSuccess ||
      cudaMemcpy(u.theta, th.data(), n * 4, cudaMemcpyHostToDevice) != cudaSuccess || repack(u, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(u.wmem);
    delete h;
    return unet_fail(ULP_ERR_CUDA, "ulp_unet_create: initialisation failed");
  }
  *out = h;
  return ULP_OK;
}

extern "C" void ulp_unet_destroy(ulp_unet net) {
  if (!net) return;
  cudaSetDevice(net->u.device);
  if (net->u.ws) cudaFree(net->u.ws);
  if (net->u.wmem) cudaFree(net->u.wmem);
  delete net;
}

extern "C" int ulp_unet_set_params(ulp_unet net, const float* params) {
  if (!net || !params) return unet_fail(ULP_ERR_INVALID, "ulp_unet_set_params: null argument");
  Unet& u = net->u;
  UCU(cudaSetDevice(u.device));
  UCU(cudaMemcpy(u.theta, params, (size_t)u.off.n * 4, cudaMemcpyHostToDevice));
  UCU(cudaMemset(u.m, 0, (size_t)u.off.n * 4));
  UCU(cudaMemset(u.v, 0, (size_t)u.off.n * 4));
  u.step = 0;
  UCU(repack(u, 0));
  UCU(cudaDeviceSynchronize());
  return ULP_OK;
}

extern "C" int ulp_unet_get_params(ulp_unet net, float* params) {
  if (!net || !params) return unet_fail(ULP_ERR_INVALID, "ulp_unet_get_params: null argument");
  Unet& u = net->u;
  UCU(cudaSetDevice(u.device));
  UCU(cudaDeviceSynchronize());
  UCU(cudaMemcpy(params, u.theta, (size_t)u.off.n * 4, cudaMemcpyDeviceToHost));
  return ULP_OK;
}

static const char kMagic[8] = {'U', 'L', 'P', 'U', 'N', 'E', 'T', '1'};

extern "C" int ulp_unet_save(ulp_unet net, const char* path) {
  if (!net || !path) return unet_fail(ULP_ERR_INVALID, "ulp_unet_save: null argument");
  std::vector<float> th((size_t)net->u.off.n);
  int rc = ulp_unet_get_params(net, th.data());
  if (rc != ULP_OK) return rc;
  FILE* f = std::fopen(path, "wb");
  if (!f) return unet_fail(ULP_ERR_INVALID, "ulp_unet_save: cannot open file");
  const long long n = net->u.off.n;
  const bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&n, sizeof(n), 1, f) == 1 &&
                  std::fwrite(th.data(), 4, th.size(), f) == th.size();
  std::fclose(f);
  return ok ? ULP_OK : unet_fail(ULP_ERR_INVALID, "ulp_unet_save: write failed");
}

extern "C" int ulp_unet_load(const char* path, ulp_unet* out) {
  if (!path || !out) return unet_fail(ULP_ERR_INVALID, "ulp_unet_load: null argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return unet_fail(ULP_ERR_INVALID, "ulp_unet_load: cannot open file");
  char mg[8];
  long long n = 0;
  const long long want = offsets().n;
  std::vector<float> th((size_t)want);
  const bool ok = std::fread(mg, 1, 8, f) == 8 && std::memcmp(mg, kMagic, 8) == 0 &&
                  std::fread(&n, sizeof(n), 1, f) == 1 && n == want &&
                  std::fread(th.data(), 4, th.size(), f) == th.size();
  std::fclose(f);
  if (!ok) return unet_fail(ULP_ERR_INVALID, "ulp_unet_load: not a parameter file of this network");
  ulp_unet h = nullptr;
  int rc = ulp_unet_create(0, &h);
  if (rc != ULP_OK) return rc;
  rc = ulp_unet_set_params(h, th.data());
  if (rc != ULP_OK) {
    ulp_unet_destroy(h);
    return rc;
  }
  *out = h;
  return ULP_OK;
}

extern "C" int ulp_unet_apply(ulp_unet net, const double* r, const double* U, const double* V, const uint8_t* mask,
                              int H, int W, double* s, void* cuda_stream) {
  if (!net || !r || !U || !V || !s) return unet_fail(ULP_ERR_INVALID, "ulp_unet_apply: null argument");
  if (H < 2 || W < 2) return unet_fail(ULP_ERR_INVALID, "ulp_unet_apply: H, W must be >= 2");
  Unet& u = net->u;
  UCU(cudaSetDevice(u.device));
  const int Hn = (H + 127) / 128 * 128, Wn = (W + 127) / 128 * 128;
  const int rc = unet_prepare(u, 1, Hn, Wn);
  if (rc) return unet_fail(rc == -5 ? ULP_ERR_NOMEM : ULP_ERR_CUDA, "ulp_unet_apply: workspace allocation failed");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  UCU(unet_apply_plane(u, r, U, V, mask, H, W, W, s, nullptr, st));
  return ULP_OK;
}

// Shared set-up of the batch entry points: offsets of B images of H x W.
static int batch_offsets(int B, const long long* pair_idx, const int* sys_idx, int H, int W, Offs& ro, Offs& uo) {
  if (B < 1 || B > kMaxBatch) return unet_fail(ULP_ERR_INVALID, "batch size must be 1..64");
  if (H % 128 || W % 128 || H < 128 || W < 128)
    return unet_fail(ULP_ERR_INVALID, "training images must be multiples of 128 in both dimensions");
  for (int b = 0; b < B; ++b) {
    const long long pi = pair_idx ? pair_idx[b] : b, si = sys_idx ? sys_idx[b] : b;
    if (pi < 0 || si < 0) return unet_fail(ULP_ERR_INVALID, "negative pair or system index");
    ro.o[b] = pi * (long long)H * W;
    uo.o[b] = si * (long long)H * W;
  }
  return ULP_OK;
}

// forward + direction loss + backward into u.grad; loss into red[kRedLoss]
static int loss_grad_impl(Unet& u, int B, const Offs& ro, const Offs& uo, int H, int W, const double* r,
                          const double* U, const double* V, const double* e, cudaStream_t st) {
  const int rc = unet_prepare(u, B, H, W);
  if (rc) return unet_fail(rc == -5 ? ULP_ERR_NOMEM : ULP_ERR_CUDA, "workspace allocation failed");
  rms(u, r, ro, B, H, W, W, u.red + kRedRho, nullptr, st);
  Src src{r, U, V, H, W, W};
  const size_t n = (size_t)B * H * W;
  k_net_in<<<eblocks(n), 256, 0, st>>>(src, ro, uo, u.red + kRedRho, B, H, W, u.xin, nullptr);
  UCU(forward(u, B, H, W, nullptr, st));
  k_head_out<<<eblocks(n), 256, 0, st>>>(u.g0, u.theta + u.off.hw, n, u.y);
  k_dir_s<<<eblocks(n), 256, 0, st>>>(src, ro, uo, u.red + kRedRho, u.y, B, u.sd);
  k_dir_stats<<<dim3(kStatBlocks, B), 256, 0, st>>>(src, ro, uo, e, u.red + kRedRho, u.sd, u.asd, u.red + kRedDir);
  k_dir_reduce<<<1, 32, 0, st>>>(u.red + kRedDir, kStatBlocks, B, u.red + kRedCoef, u.red + kRedLoss);
  k_dir_grad<<<eblocks(n), 256, 0, st>>>(src, ro, u.red + kRedRho, u.asd, u.red + kRedCoef, B, u.t);
  UCU(backward(u, B, H, W, st));
  return ULP_OK;
}

extern "C" int ulp_unet_forward(ulp_unet net, int B, int H, int W, const double* r, const double* U, const double* V,
                                float* y, void* cuda_stream) {
  if (!net || !r || !U || !V || !y) return unet_fail(ULP_ERR_INVALID, "ulp_unet_forward: null argument");
  Unet& u = net->u;
  UCU(cudaSetDevice(u.device));
  Offs ro{}, uo{};
  int rc = batch_offsets(B, nullptr, nullptr, H, W, ro, uo);
  if (rc != ULP_OK) return rc;
  rc = unet_prepare(u, B, H, W);
  if (rc) return unet_fail(rc == -5 ? ULP_ERR_NOMEM : ULP_ERR_CUDA, "workspace allocation failed");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rms(u, r, ro, B, H, W, W, u.red + kRedRho, nullptr, st);
  Src src{r, U, V, H, W, W};
  k_net_in<<<eblocks((size_t)B * H * W), 256, 0, st>>>(src, ro, uo, u.red + kRedRho, B, H, W, u.xin, nullptr);
  UCU(forward(u, B, H, W, nullptr, st));
  const size_t n = (size_t)B * H * W;
  k_head_out<<<eblocks(n), 256, 0, st>>>(u.g0, u.theta + u.off.hw, n, y);
  UCU(cudaGetLastError());
  return ULP_OK;
}

extern "C" int ulp_unet_loss_grad(ulp_unet net, int B, int H, int W, const double* r, const double* U,
                                  const double* V, const double* e, double* loss, float* grad, void* cuda_stream) {
  if (!net || !r || !U || !V || !e) return unet_fail(ULP_ERR_INVALID, "ulp_unet_loss_grad: null argument");
  Unet& u = net->u;
  UCU(cudaSetDevice(u.device));
  Offs ro{}, uo{};
  int rc = batch_offsets(B, nullptr, nullptr, H, W, ro, uo);
  if (rc != ULP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rc = loss_grad_impl(u, B, ro, uo, H, W, r, U, V, e, st);
  if (rc != ULP_OK) return rc;
  if (grad) UCU(cudaMemcpyAsync(grad, u.grad, (size_t)u.off.n * 4, cudaMemcpyDeviceToDevice, st));
  if (loss) {
    UCU(cudaMemcpyAsync(loss, u.red + kRedLoss, sizeof(double), cudaMemcpyDeviceToHost, st));
    UCU(cudaStreamSynchronize(st));
  }
  if (unet_error(u)) return unet_fail(ULP_ERR_TIMEOUT, "ulp_unet_loss_grad: a tensor-core wait timed out");
  return ULP_OK;
}

extern "C" int ulp_unet_train_step(ulp_unet net, int B, const long long* pair_idx, const int* sys_idx, int H, int W,
                                   const double* r, const double* e, const double* U, const double* V, float lr,
                                   double* loss, void* cuda_stream) {
  if (!net || !pair_idx || !sys_idx || !r || !e || !U || !V)
    return unet_fail(ULP_ERR_INVALID, "ulp_unet_train_step: null argument");
  if (!(lr > 0.f)) return unet_fail(ULP_ERR_INVALID, "ulp_unet_train_step: lr must be > 0");
  Unet& u = net->u;
  UCU(cudaSetDevice(u.device));
  Offs ro{}, uo{};
  int rc = batch_offsets(B, pair_idx, sys_idx, H, W, ro, uo);
  if (rc != ULP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rc = loss_grad_impl(u, B, ro, uo, H, W, r, U, V, e, st);
  if (rc != ULP_OK) return rc;
  u.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)u.step), c2 = 1.f - std::pow(b2, (float)u.step);
  k_adam<<<eblocks((size_t)u.off.n), 256, 0, st>>>(u.theta, u.grad, u.m, u.v, u.off.n, lr, b1, b2, 1e-8f, c1, c2);
  UCU(repack(u, st));
  if (loss) {
    UCU(cudaMemcpyAsync(loss, u.red + kRedLoss, sizeof(double), cudaMemcpyDeviceToHost, st));
    UCU(cudaStreamSynchronize(st));
    if (unet_error(u)) return unet_fail(ULP_ERR_TIMEOUT, "ulp_unet_train_step: a tensor-core wait timed out");
  }
  return ULP_OK;
}

// ------------------------------------------------------------------ training pairs
namespace ulp {
namespace unet {
__global__ void k_pair(const double* __restrict__ b, const double* __restrict__ aphi, const double* __restrict__ phis,
                       const double* __restrict__ phil, size_t n, double* __restrict__ r, double* __restrict__ e) {
  GRID_STRIDE(t, n) {
    r[t] = b[t] - aphi[t];
    e[t] = phis[t] - phil[t];
  }
}
}  // namespace unet
}  // namespace ulp

extern "C" int ulp_unet_harvest(const double* U, const double* V, const double* b, int H, int W, int precond,
                                double tol_star, int n, const int* iters, double* r_out, double* e_out,
                                void* cuda_stream) {
  if (!U || !V || !b || !iters || !r_out || !e_out || n < 1)
    return unet_fail(ULP_ERR_INVALID, "ulp_unet_harvest: null argument or n < 1");
  if (precond != ULP_PRECOND_IDENTITY && precond != ULP_PRECOND_JACOBI)
    return unet_fail(ULP_ERR_UNSUPPORTED, "ulp_unet_harvest: identity or Jacobi PCG only");
  if (!(tol_star > 0.0)) return unet_fail(ULP_ERR_INVALID, "ulp_unet_harvest: tol_star must be > 0");
  for (int k = 0; k < n; ++k)
    if (iters[k] < 0) return unet_fail(ULP_ERR_INVALID, "ulp_unet_harvest: negative iteration count");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t hw = (size_t)H * W;
  double* buf = nullptr;
  UCU(cudaMalloc(&buf, 3 * hw * sizeof(double)));
  double *phis = buf, *phil = buf + hw, *aphi = buf + 2 * hw;
  // one plan for every solve of the harvest (its flexible-CG graph is built once)
  ulp_plan plan = nullptr;
  int rc = ulp_plan_create(H, W, nullptr, &plan);
  ulp_stats s;
  // phi*: the multigrid flexible-CG solution (the same system and tolerance, reached in tens of
  // iterations instead of the thousands a plain PCG needs at tol_star)
  if (rc == ULP_OK && cudaMemsetAsync(phis, 0, hw * sizeof(double), st) != cudaSuccess) rc = ULP_ERR_CUDA;
  if (rc == ULP_OK) rc = pcg_on_plan(plan, U, V, b, ULP_PRECOND_MG, tol_star, 0, phis, st, &s);
  if (rc > 0) rc = ULP_OK;  // not converged to tol_star within l_max: the iterate is still the best estimate
  for (int k = 0; k < n && rc == ULP_OK; ++k) {
    if (cudaMemsetAsync(phil, 0, hw * sizeof(double), st) != cudaSuccess) rc = ULP_ERR_CUDA;
    if (rc == ULP_OK && iters[k] > 0) {
      rc = pcg_on_plan(plan, U, V, b, precond, 1e-300, iters[k], phil, st, &s);
      if (rc > 0) rc = ULP_OK;
    }
    if (rc == ULP_OK) rc = matvec_on_plan(plan, U, V, phil, aphi, st);
    if (rc == ULP_OK) {
      unet::k_pair<<<(int)((hw + 255) / 256 < 4096 ? (hw + 255) / 256 : 4096), 256, 0, st>>>(b, aphi, phis, phil, hw, r_out + k * hw, e_out + k * hw);
      if (cudaGetLastError() != cudaSuccess) rc = ULP_ERR_CUDA;
    }
  }
  cudaStreamSynchronize(st);
  if (plan) ulp_plan_destroy(plan);
  cudaFree(buf);
  return rc == ULP_OK ? ULP_OK : (rc == ULP_ERR_CUDA ? unet_fail(ULP_ERR_CUDA, "ulp_unet_harvest: CUDA error") : rc);
}
