// ulp_dct.cu -- DCT Poisson preconditioner on the 5th-generation tensor cores.
//
// s = Pi L^+ r, L the unit-weight Neumann 5-point Laplacian (the Fourier /
// Green-function approach the paper cites in Sec. 1): its eigenvectors are
// products of orthonormal DCT-II vectors with eigenvalues
// (2 - 2 cos(pi a / H)) + (2 - 2 cos(pi b / W)), so with C_n the n x n DCT-II
// matrix
//     R^ = C_H R C_W^T,   S^ = R^ / Lambda (zero mode dropped),   S = C_H^T S^ C_W,
// and Pi zeroes masked pixels.  The four products are dense contractions and
// run as BF16 tcgen05 GEMMs with FP32 accumulation in tensor memory.
//
// Split-BF16 operands: every operand X is held as two BF16 planes, X = Xh + Xl
// with Xh = bf16(X) and Xl = bf16(X - Xh) (16 significant bits together), and
// each product is A B^T ~ Ah Bh^T + Ah Bl^T + Al Bh^T: one GEMM over three
// K-segments, the TMA producer loading (Ah, Bh), (Ah, Bl), (Al, Bh) in turn into
// the same accumulator.  The dropped Al Bl^T term and the residual of the split
// are about 2^-16 of each product, so one application is within about 4e-5 of
// the exact operator (plain BF16 operands: about 1e-2).  Every epilogue that
// feeds the next GEMM writes both planes of its output.
//
// GEMM form: C[m][n] = sum_k A[m][k] B[n][k] with both operands K-major
// (row-major, k contiguous), BM = 128, BN = 128, BK = 64 (one 128-byte
// swizzle atom of BF16 per row), operands staged by TMA into a 3-stage ring,
// one elected thread issuing tcgen05.mma, the accumulator read back by all
// four warps with tcgen05.ld.  The epilogue stores C transposed, out[n][m]:
// a warp holds 32 consecutive m of one n, so the transposed store is the
// coalesced one, and four transposed GEMMs chain without a transpose pass:
//   G1  A = R (i,j)     B = C_W (b,j)    -> X^T  (b,i)
//   G2  A = X^T (b,i)   B = C_H (a,i)    -> R^ (a,b), times 1/Lambda(a,b)
//   G3  A = S^ (a,b)    B = C_W^T (j,b)  -> Y^T  (j,a)
//   G4  A = Y^T (j,a)   B = C_H^T (i,a)  -> S (i,j), masked, FP64 into the plane
// Every wait is bounded; on a time-out the kernel records an error, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "ulp_host.h"
#include "ulp_tc.cuh"

namespace ulp {

constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 3;
constexpr int kTileBytes = kBM * kBK * 2;                 // 16 KB per operand tile
constexpr int kStageBytes = 2 * kTileBytes;               // A + B
constexpr int kGemmSmem = kStages * kStageBytes + 1024 + 256 + 512;  // + alignment + barriers + 1/Lambda rows

enum Epi { kEpiBf16T = 0, kEpiBf16TScale = 1, kEpiF64TMask = 2 };

struct GemmOut {
  void* out;           // Epi 0/1: bf16 [N][ldo]; Epi 2: double plane [*][ldo]
  void* out_lo;        // Epi 0/1: the low BF16 plane of the split output, same layout
  int ldo;
  const float* lh;     // Epi 1: eigenvalues 2 - 2 cos(pi a / H) by output row n (+inf on padding)
  const float* lw;     // Epi 1: eigenvalues 2 - 2 cos(pi b / W) by output column m (+inf on padding)
  const unsigned* mbits; // Epi 2: mask bits, bit (n & 31) of word [n >> 5][m] (1 = zero the output), or null
  int ldb;               // Epi 2: row stride of mbits in words
  int rows, cols;      // Epi 2: only n < rows and m < cols are written
  int* err;
};

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

// tmA / tmB: the high planes, tmAl / tmBl: the low planes; K-segments (Ah, Bh), (Ah, Bl),
// (Al, Bh) in that order, all accumulated into one tensor-memory tile
template <int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm_nt(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB,
                                                    const __grid_constant__ CUtensorMap tmAl,
                                                    const __grid_constant__ CUtensorMap tmBl, int K, GemmOut o) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int nkb0 = K / kBK, nkb = 3 * nkb0;  // three K-segments of the split product
  float* s_lh = reinterpret_cast<float*>(base + kStages * kStageBytes + 256);
  const int m = m0 + warp * 32 + lane;  // this thread's accumulator row in the epilogue
  float lwm = 0.f;
  uint32_t zbits[kBN / 32] = {};        // Epi 2: mask bits of this thread's 128 outputs
  if (EPI == kEpiBf16TScale) {
    s_lh[threadIdx.x] = o.lh[n0 + threadIdx.x];
    lwm = o.lw[m];
  } else if (EPI == kEpiF64TMask) {
    // four coalesced words, issued before the main loop so they overlap the MMAs
    if (o.mbits) {
#pragma unroll
      for (int w = 0; w < kBN / 32; ++w) zbits[w] = __ldg(o.mbits + (size_t)((n0 >> 5) + w) * o.ldb + m);
    }
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kStages, u = kb / kStages;
      if (u > 0 && !mbar_wait(empty + s, (u - 1) & 1, o.err)) break;
      unsigned char* sa = base + s * kStageBytes;
      const int seg = kb / nkb0, kc = (kb - seg * nkb0) * kBK;
      mbar_expect_tx(full + s, kStageBytes);
      tma_load_2d(sa, seg == 2 ? &tmAl : &tmA, full + s, kc, m0);
      tma_load_2d(sa + kTileBytes, seg == 1 ? &tmBl : &tmB, full + s, kc, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: four K = 16 steps per 64-wide stage, advancing the descriptors by 32 bytes
    bool ok = true;
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int s = kb % kStages, u = kb / kStages;
      if (!mbar_wait(full + s, u & 1, o.err)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned char* sa = base + s * kStageBytes;
      const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + kTileBytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        mma_bf16(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), kIdesc, (kb | kk) != 0);
      mma_commit(empty + s);
    }
    mma_commit(done);
  }
  __syncwarp();

  // epilogue: warp w owns accumulator lanes (rows m) 32w .. 32w+31
  const bool ready = __all_sync(0xffffffffu, mbar_wait(done, 0, o.err));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready) {
#pragma unroll 1
    for (int c = 0; c < kBN / 16; ++c) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int n = n0 + c * 16 + q;
        const size_t off = (size_t)n * o.ldo + m;
        if (EPI == kEpiBf16T || EPI == kEpiBf16TScale) {
          float w = v[q];
          // 1/Lambda(a, b) with a = n, b = m; the zero mode and the padding give 0
          if (EPI == kEpiBf16TScale) w *= (n | m) ? 1.f / (s_lh[c * 16 + q] + lwm) : 0.f;
          const __nv_bfloat16 h = __float2bfloat16_rn(w);
          reinterpret_cast<__nv_bfloat16*>(o.out)[off] = h;
          reinterpret_cast<__nv_bfloat16*>(o.out_lo)[off] = __float2bfloat16_rn(w - __bfloat162float(h));
        } else {
          if (n < o.rows && m < o.cols) {
            const int nn = c * 16 + q;
            const bool z = (zbits[nn >> 5] >> (nn & 31)) & 1u;
            reinterpret_cast<double*>(o.out)[off] = z ? 0.0 : (double)v[q];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBN));
}

// r (FP64 plane) -> R = Rh + Rl (split BF16, Hp x Wp, zero padding)
__global__ void k_pack_bf16(const double* __restrict__ r, int H, int W, int pitch, __nv_bfloat16* R,
                            __nv_bfloat16* Rl, int Hp, int Wp) {
  const size_t n = (size_t)Hp * Wp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / Wp), j = (int)(t % Wp);
    const float v = (i < H && j < W) ? (float)r[(size_t)i * pitch + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    R[t] = h;
    Rl[t] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// mask (uint8 plane, pitch) -> bits[(i >> 5)][j], bit (i & 31); rows >= H and columns >= W are 0
__global__ void k_mask_bits(const uint8_t* __restrict__ mask, int H, int W, int pitch, unsigned* bits, int Hp,
                            int Wp) {
  const int nw = Hp / 32;
  const size_t n = (size_t)nw * Wp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int w = (int)(t / Wp), j = (int)(t % Wp);
    unsigned v = 0;
    if (j < W)
      for (int b = 0; b < 32; ++b) {
        const int i = 32 * w + b;
        if (i < H && mask[(size_t)i * pitch + j]) v |= 1u << b;
      }
    bits[t] = v;
  }
}

// ------------------------------------------------------------------ host side
// 2-D BF16 tensor [rows][cols] (cols contiguous), box 64 x 128, 128-byte swizzle.
static bool make_map(CUtensorMap* tm, const void* ptr, int rows, int cols) {
  PFN_encodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// dynamic shared memory above 48 KB is an attribute of the function on the current device:
// set when a plan is made on it
static void gemm_attrs() {
  cudaFuncSetAttribute(k_gemm_nt<kEpiBf16T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  cudaFuncSetAttribute(k_gemm_nt<kEpiBf16TScale>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  cudaFuncSetAttribute(k_gemm_nt<kEpiF64TMask>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
}

// A split operand: its high and low BF16 planes.
struct Split {
  const void* h;
  const void* l;
};

template <int EPI>
static cudaError_t gemm(Split A, int M, Split B, int N, int K, const GemmOut& o, cudaStream_t st) {
  CUtensorMap ta, tb, tal, tbl;
  if (!make_map(&ta, A.h, M, K) || !make_map(&tb, B.h, N, K) || !make_map(&tal, A.l, M, K) ||
      !make_map(&tbl, B.l, N, K))
    return cudaErrorInvalidValue;
  dim3 grid(N / kBN, M / kBM);
  k_gemm_nt<EPI><<<grid, 128, kGemmSmem, st>>>(ta, tb, tal, tbl, K, o);
  return cudaGetLastError();
}

// Orthonormal DCT-II matrix of size n padded to np, C[k][x] = c_k cos(pi k (x + 1/2) / n),
// as split BF16 (high, low) planes, and its transpose.
static void dct_matrix(int n, int np, std::vector<__nv_bfloat16>& C, std::vector<__nv_bfloat16>& Cl,
                       std::vector<__nv_bfloat16>& CT, std::vector<__nv_bfloat16>& CTl) {
  for (auto* v : {&C, &Cl, &CT, &CTl}) v->assign((size_t)np * np, __float2bfloat16(0.f));
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double ck = (k == 0) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    for (int x = 0; x < n; ++x) {
      const double c = ck * std::cos(pi * k * (x + 0.5) / n);
      const __nv_bfloat16 h = __float2bfloat16((float)c);
      const __nv_bfloat16 l = __float2bfloat16((float)(c - (double)__bfloat162float(h)));
      C[(size_t)k * np + x] = h;
      Cl[(size_t)k * np + x] = l;
      CT[(size_t)x * np + k] = h;
      CTl[(size_t)x * np + k] = l;
    }
  }
}

// Device buffers of the DCT preconditioner for an H x W map (allocated with the plan).
struct DctPlan {
  int H = 0, W = 0, Hp = 0, Wp = 0;
  __nv_bfloat16 *CH = nullptr, *CHT = nullptr, *CW = nullptr, *CWT = nullptr;      // high planes
  __nv_bfloat16 *CHl = nullptr, *CHTl = nullptr, *CWl = nullptr, *CWTl = nullptr;  // low planes
  __nv_bfloat16 *R = nullptr, *X = nullptr, *Y = nullptr;     // R, X^T / S^, Y^T (high)
  __nv_bfloat16 *Rl = nullptr, *Xl = nullptr, *Yl = nullptr;  // their low planes
  float *lh = nullptr, *lw = nullptr;                        // [Hp], [Wp] eigenvalue factors
  unsigned* mbits = nullptr;                                 // [Hp / 32][Wp] mask bits
  int* err = nullptr;
  void* mem = nullptr;
};

size_t dct_bytes(int H, int W) {
  const size_t Hp = (H + 127) / 128 * 128, Wp = (W + 127) / 128 * 128;
  return 2 * 2 * (Hp * Hp + Wp * Wp) * 2 + 2 * 3 * Hp * Wp * 2 + (Hp + Wp) * 4 + Hp / 32 * Wp * 4 + 8192;
}

// Builds the matrices into mem (dct_bytes(H, W) bytes of device memory).
int dct_setup(DctPlan& d, int H, int W, void* mem) {
  d.H = H;
  d.W = W;
  d.Hp = (H + 127) / 128 * 128;
  d.Wp = (W + 127) / 128 * 128;
  d.mem = mem;
  char* p = static_cast<char*>(mem);
  auto take = [&](size_t bytes) {
    void* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  const size_t Hp = d.Hp, Wp = d.Wp;
  d.CH = static_cast<__nv_bfloat16*>(take(Hp * Hp * 2));
  d.CHT = static_cast<__nv_bfloat16*>(take(Hp * Hp * 2));
  d.CW = static_cast<__nv_bfloat16*>(take(Wp * Wp * 2));
  d.CWT = static_cast<__nv_bfloat16*>(take(Wp * Wp * 2));
  d.CHl = static_cast<__nv_bfloat16*>(take(Hp * Hp * 2));
  d.CHTl = static_cast<__nv_bfloat16*>(take(Hp * Hp * 2));
  d.CWl = static_cast<__nv_bfloat16*>(take(Wp * Wp * 2));
  d.CWTl = static_cast<__nv_bfloat16*>(take(Wp * Wp * 2));
  d.R = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.X = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.Y = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.Rl = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.Xl = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.Yl = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.lh = static_cast<float*>(take(Hp * 4));
  d.lw = static_cast<float*>(take(Wp * 4));
  d.mbits = static_cast<unsigned*>(take(Hp / 32 * Wp * 4));
  d.err = static_cast<int*>(take(256));
  std::vector<__nv_bfloat16> C, Cl, CT, CTl;
  auto up = [](void* dst, const std::vector<__nv_bfloat16>& v) {
    return cudaMemcpy(dst, v.data(), v.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  dct_matrix(H, d.Hp, C, Cl, CT, CTl);
  if (!up(d.CH, C) || !up(d.CHl, Cl) || !up(d.CHT, CT) || !up(d.CHTl, CTl)) return -2;
  dct_matrix(W, d.Wp, C, Cl, CT, CTl);
  if (!up(d.CW, C) || !up(d.CWl, Cl) || !up(d.CWT, CT) || !up(d.CWTl, CTl)) return -2;
  // the split copy of r starts at zero: the flexible CG writes only its H x W part, and the
  // GEMMs multiply the padding by the matrices' zero padding (which must not meet a NaN pattern)
  if (cudaMemset(d.R, 0, Hp * Wp * 2) != cudaSuccess || cudaMemset(d.Rl, 0, Hp * Wp * 2) != cudaSuccess) return -2;
  // Lambda(a, b) = lh[a] + lw[b]; padded indices get +inf so that 1/Lambda = 0 there
  const double pi = 3.14159265358979323846;
  std::vector<float> lh(Hp, INFINITY), lw(Wp, INFINITY);
  for (int a = 0; a < H; ++a) lh[a] = (float)(2.0 - 2.0 * std::cos(pi * a / H));
  for (int b = 0; b < W; ++b) lw[b] = (float)(2.0 - 2.0 * std::cos(pi * b / W));
  if (cudaMemcpy(d.lh, lh.data(), Hp * 4, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
  if (cudaMemcpy(d.lw, lw.data(), Wp * 4, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
  if (cudaMemset(d.err, 0, 256) != cudaSuccess) return -2;
  return 0;
}

DctPlan* dct_create(int H, int W, void* mem) {
  gemm_attrs();
  DctPlan* d = new DctPlan();
  if (dct_setup(*d, H, W, mem) != 0) {
    delete d;
    return nullptr;
  }
  return d;
}

void dct_destroy(DctPlan* d) { delete d; }

int dct_error(const DctPlan& d) {
  int e = 0;
  cudaMemcpy(&e, d.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) cudaMemset(d.err, 0, sizeof(int));
  return e;
}

// s = Pi L^+ r: r, s are FP64 planes with the given pitch; mask a uint8 plane or null.
unsigned* dct_input(const DctPlan& d, int* ld_pairs, unsigned** lo) {
  *ld_pairs = d.Wp / 2;
  *lo = reinterpret_cast<unsigned*>(d.Rl);
  return reinterpret_cast<unsigned*>(d.R);
}

static int elem_blocks(size_t n) { return (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048); }

cudaError_t dct_prepare_mask(const DctPlan& d, const uint8_t* mask, int pitch, cudaStream_t st) {
  if (mask)
    k_mask_bits<<<elem_blocks((size_t)d.Hp / 32 * d.Wp), 256, 0, st>>>(mask, d.H, d.W, pitch, d.mbits, d.Hp, d.Wp);
  return cudaGetLastError();
}

cudaError_t dct_apply(const DctPlan& d, const double* r, int pitch, const uint8_t* mask, double* s,
                      cudaStream_t st, bool packed) {
  const int Hp = d.Hp, Wp = d.Wp;
  if (!packed) {
    k_pack_bf16<<<elem_blocks((size_t)Hp * Wp), 256, 0, st>>>(r, d.H, d.W, pitch, d.R, d.Rl, Hp, Wp);
    const cudaError_t e = dct_prepare_mask(d, mask, pitch, st);
    if (e != cudaSuccess) return e;
  }
  GemmOut o{};
  o.err = d.err;
  // G1: X^T[b][i] = sum_j R[i][j] C_W[b][j]
  o.out = d.X;
  o.out_lo = d.Xl;
  o.ldo = Hp;
  cudaError_t e = gemm<kEpiBf16T>({d.R, d.Rl}, Hp, {d.CW, d.CWl}, Wp, Wp, o, st);
  if (e != cudaSuccess) return e;
  // G2: S^[a][b] = (sum_i X^T[b][i] C_H[a][i]) / Lambda[a][b]
  o.out = d.Y;
  o.out_lo = d.Yl;
  o.ldo = Wp;
  o.lh = d.lh;
  o.lw = d.lw;
  e = gemm<kEpiBf16TScale>({d.X, d.Xl}, Wp, {d.CH, d.CHl}, Hp, Hp, o, st);
  if (e != cudaSuccess) return e;
  // G3: Y^T[j][a] = sum_b S^[a][b] C_W^T[j][b]
  o.out = d.X;
  o.out_lo = d.Xl;
  o.ldo = Hp;
  o.lh = o.lw = nullptr;
  e = gemm<kEpiBf16T>({d.Y, d.Yl}, Hp, {d.CWT, d.CWTl}, Wp, Wp, o, st);
  if (e != cudaSuccess) return e;
  // G4: S[i][j] = sum_a Y^T[j][a] C_H^T[i][a], masked, into the FP64 plane
  o.out = s;
  o.out_lo = nullptr;
  o.ldo = pitch;
  o.mbits = mask ? d.mbits : nullptr;
  o.ldb = Wp;
  o.rows = d.H;
  o.cols = d.W;
  return gemm<kEpiF64TMask>({d.X, d.Xl}, Wp, {d.CHT, d.CHTl}, Hp, Hp, o, st);
}

}  // namespace ulp
