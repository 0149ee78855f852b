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

namespace ulp {

constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 3;
constexpr int kTileBytes = kBM * kBK * 2;                 // 16 KB per operand tile
constexpr int kStageBytes = 2 * kTileBytes;               // A + B
constexpr int kGemmSmem = kStages * kStageBytes + 1024 + 256;  // + alignment + barriers

enum Epi { kEpiBf16T = 0, kEpiBf16TScale = 1, kEpiF64TMask = 2 };

struct GemmOut {
  void* out;           // Epi 0/1: bf16 [N][ldo]; Epi 2: double plane [*][ldo]
  int ldo;
  const float* scale;  // Epi 1: [N][ldo] multiplier
  const uint8_t* mask; // Epi 2: [*][ldo] (1 = zero the output), may be null
  int rows, cols;      // Epi 2: only n < rows and m < cols are written
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false (and the error flag set) after 2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*(volatile int*)err || globaltimer() - t0 > 2000000000ull) {
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  // shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
  // 1024 bytes (stride byte offset), descriptor version 1
  const uint64_t a = (smem_u32(p) & 0x3FFFFu) >> 4;
  return a | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

template <int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm_nt(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, int K, GemmOut o) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int nkb = K / kBK;

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
      mbar_expect_tx(full + s, kStageBytes);
      tma_load_2d(sa, &tmA, full + s, kb * kBK, m0);
      tma_load_2d(sa + kTileBytes, &tmB, full + s, kb * kBK, n0);
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
    const int m = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < kBN / 16; ++c) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int n = n0 + c * 16 + q;
        const size_t off = (size_t)n * o.ldo + m;
        if (EPI == kEpiBf16T) {
          reinterpret_cast<__nv_bfloat16*>(o.out)[off] = __float2bfloat16_rn(v[q]);
        } else if (EPI == kEpiBf16TScale) {
          reinterpret_cast<__nv_bfloat16*>(o.out)[off] = __float2bfloat16_rn(v[q] * o.scale[off]);
        } else {
          if (n < o.rows && m < o.cols) {
            const bool z = o.mask && o.mask[off];
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

// r (FP64 plane) -> R (BF16, Hp x Wp, zero padding)
__global__ void k_pack_bf16(const double* __restrict__ r, int H, int W, int pitch, __nv_bfloat16* R, int Hp,
                            int Wp) {
  const size_t n = (size_t)Hp * Wp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / Wp), j = (int)(t % Wp);
    R[t] = __float2bfloat16_rn((i < H && j < W) ? (float)r[(size_t)i * pitch + j] : 0.f);
  }
}

// ------------------------------------------------------------------ host side
using PFN_encodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                     CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                     CUtensorMapFloatOOBfill);

static PFN_encodeTiled encode_fn() {
  static PFN_encodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(p);
  }
  return fn;
}

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

template <int EPI>
static cudaError_t gemm(const void* A, int M, const void* B, int N, int K, const GemmOut& o, cudaStream_t st) {
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, M, K) || !make_map(&tb, B, N, K)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_nt<kEpiBf16T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    cudaFuncSetAttribute(k_gemm_nt<kEpiBf16TScale>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    cudaFuncSetAttribute(k_gemm_nt<kEpiF64TMask>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    attr = true;
  }
  dim3 grid(N / kBN, M / kBM);
  k_gemm_nt<EPI><<<grid, 128, kGemmSmem, st>>>(ta, tb, K, o);
  return cudaGetLastError();
}

// Orthonormal DCT-II matrix of size n padded to np: C[k][x] = c_k cos(pi k (x + 1/2) / n).
static void dct_matrix(int n, int np, std::vector<__nv_bfloat16>& C, std::vector<__nv_bfloat16>& CT) {
  C.assign((size_t)np * np, __float2bfloat16(0.f));
  CT.assign((size_t)np * np, __float2bfloat16(0.f));
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double ck = (k == 0) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    for (int x = 0; x < n; ++x) {
      const __nv_bfloat16 v = __float2bfloat16((float)(ck * std::cos(pi * k * (x + 0.5) / n)));
      C[(size_t)k * np + x] = v;
      CT[(size_t)x * np + k] = v;
    }
  }
}

// Device buffers of the DCT preconditioner for an H x W map (allocated with the plan).
struct DctPlan {
  int H = 0, W = 0, Hp = 0, Wp = 0;
  __nv_bfloat16 *CH = nullptr, *CHT = nullptr, *CW = nullptr, *CWT = nullptr;
  __nv_bfloat16 *R = nullptr, *X = nullptr, *Y = nullptr;  // R, X^T / S^, Y^T
  float* lam_inv = nullptr;                                  // [Hp][Wp]
  int* err = nullptr;
  void* mem = nullptr;
};

size_t dct_bytes(int H, int W) {
  const size_t Hp = (H + 127) / 128 * 128, Wp = (W + 127) / 128 * 128;
  return 2 * (Hp * Hp + Wp * Wp) * 2 + 3 * Hp * Wp * 2 + Hp * Wp * 4 + 4096;
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
  d.R = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.X = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.Y = static_cast<__nv_bfloat16*>(take(Hp * Wp * 2));
  d.lam_inv = static_cast<float*>(take(Hp * Wp * 4));
  d.err = static_cast<int*>(take(256));
  std::vector<__nv_bfloat16> C, CT;
  dct_matrix(H, d.Hp, C, CT);
  if (cudaMemcpy(d.CH, C.data(), C.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
  if (cudaMemcpy(d.CHT, CT.data(), CT.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
  dct_matrix(W, d.Wp, C, CT);
  if (cudaMemcpy(d.CW, C.data(), C.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
  if (cudaMemcpy(d.CWT, CT.data(), CT.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
  std::vector<float> li(Hp * Wp, 0.f);
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < W; ++b) {
      if (a == 0 && b == 0) continue;
      const double lam = (2.0 - 2.0 * std::cos(pi * a / H)) + (2.0 - 2.0 * std::cos(pi * b / W));
      li[(size_t)a * Wp + b] = (float)(1.0 / lam);
    }
  if (cudaMemcpy(d.lam_inv, li.data(), li.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
  if (cudaMemset(d.err, 0, 256) != cudaSuccess) return -2;
  return 0;
}

DctPlan* dct_create(int H, int W, void* mem) {
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
cudaError_t dct_apply(const DctPlan& d, const double* r, int pitch, const uint8_t* mask, double* s,
                      cudaStream_t st) {
  const int Hp = d.Hp, Wp = d.Wp;
  k_pack_bf16<<<(Hp * Wp + 255) / 256 < 2048 ? (Hp * Wp + 255) / 256 : 2048, 256, 0, st>>>(r, d.H, d.W, pitch,
                                                                                         d.R, Hp, Wp);
  GemmOut o{};
  o.err = d.err;
  // G1: X^T[b][i] = sum_j R[i][j] C_W[b][j]
  o.out = d.X;
  o.ldo = Hp;
  cudaError_t e = gemm<kEpiBf16T>(d.R, Hp, d.CW, Wp, Wp, o, st);
  if (e != cudaSuccess) return e;
  // G2: S^[a][b] = (sum_i X^T[b][i] C_H[a][i]) / Lambda[a][b]
  o.out = d.Y;
  o.ldo = Wp;
  o.scale = d.lam_inv;
  e = gemm<kEpiBf16TScale>(d.X, Wp, d.CH, Hp, Hp, o, st);
  if (e != cudaSuccess) return e;
  // G3: Y^T[j][a] = sum_b S^[a][b] C_W^T[j][b]
  o.out = d.X;
  o.ldo = Hp;
  o.scale = nullptr;
  e = gemm<kEpiBf16T>(d.Y, Hp, d.CWT, Wp, Wp, o, st);
  if (e != cudaSuccess) return e;
  // G4: S[i][j] = sum_a Y^T[j][a] C_H^T[i][a], masked, into the FP64 plane
  o.out = s;
  o.ldo = pitch;
  o.mask = mask;
  o.rows = d.H;
  o.cols = d.W;
  return gemm<kEpiF64TMask>(d.X, Wp, d.CHT, Hp, Hp, o, st);
}

}  // namespace ulp
