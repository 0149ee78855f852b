// ulp_noalloc.cu -- ulp_pcg_noalloc: the inner PCG solve of ulp_pcg for
// callers that cannot allocate device memory.  All workspace lives in one
// file-scope static device array; nothing is allocated or freed per call.
//
// Who needs this: a caller whose device memory is already owned by another
// allocator (a framework's caching pool that reserved the free memory, where a
// cudaMalloc would fail or force the pool to give memory back), and a caller on
// a latency-bound loop that cannot pay for cudaMalloc/cudaFree (cudaFree waits
// for the whole device) or cannot risk an out-of-memory error in mid-run.
// ulp_pcg builds and frees a temporary plan on every call, so it serves
// neither.
//
// Limits and sharing: the array holds one map of at most kNoAllocElems padded
// elements (H rows x W rounded up to 64 columns); every GPU that loads this
// library keeps the array until the process exits.  Every call on a device
// uses the same array and leaves its contents behind; each call clears the
// part it uses before use.  Calls whose work overlaps on the GPU (other
// streams, or other host threads) race on the array and must be serialised
// by the caller.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ulp_host.h"

namespace ulp {
namespace {

constexpr size_t kNoAllocElems = 65536;                // e.g. 256 x 256, 128 x 512
constexpr size_t kPlanes = 14;                         // FP64 planes used by the PCG path
constexpr size_t kNoAllocBytes = 8u << 20;             // 8 MiB

__device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Per-device set-up: the array's device address, SM count and solver occupancy.
struct DeviceSetup {
  bool ready = false;
  void* base = nullptr;
  int nsm = 0;
  int bps = 0;
  Plan plan;  // host description of the layout inside the array (one map)
};
constexpr int kMaxDevices = 64;
DeviceSetup g_dev[kMaxDevices];
std::mutex g_mu;

__global__ void k_store_map(MapDesc M, MapDesc* dst) { *dst = M; }

int nfail(int code, const char* msg) { return set_error(code, msg); }

}  // namespace
}  // namespace ulp

using namespace ulp;

extern "C" int ulp_pcg_noalloc(const double* U, const double* V, const double* b, int H, int W,
                               int precond, double tol, int max_inner, double* phi, void* cuda_stream,
                               ulp_stats* stats) {
  if (!U || !V || !b || !phi) return nfail(ULP_ERR_INVALID, "ulp_pcg_noalloc: null argument");
  if (H < 2 || W < 2) return nfail(ULP_ERR_INVALID, "ulp_pcg_noalloc: H and W must be >= 2");
  const size_t pitch = ((size_t)W + kStrip - 1) / kStrip * kStrip;
  if ((size_t)H * pitch > kNoAllocElems)
    return nfail(ULP_ERR_INVALID,
                 "ulp_pcg_noalloc: grid too large for the static workspace "
                 "(H * round_up(W, 64) must be <= 65536, e.g. 256 x 256)");
  if (precond != ULP_PRECOND_IDENTITY && precond != ULP_PRECOND_JACOBI)
    return nfail(ULP_ERR_UNSUPPORTED, "ulp_pcg_noalloc: only ULP_PRECOND_IDENTITY and ULP_PRECOND_JACOBI");
  if (!(tol > 0.0)) return nfail(ULP_ERR_INVALID, "ulp_pcg_noalloc: tol must be > 0");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return nfail(ULP_ERR_CUDA, "ulp_pcg_noalloc: no usable current device");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSetup& D = g_dev[dev];
  if (!D.ready) {
    // First call on this device (the device is current): find the array's
    // device address.  The name g_scratch in host code is only a stand-in.
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return nfail(ULP_ERR_CUDA, "ulp_pcg_noalloc: cudaGetSymbolAddress failed");
    }
    int coop = 0;
    if (cudaDeviceGetAttribute(&D.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
      return nfail(ULP_ERR_CUDA, "ulp_pcg_noalloc: device attributes unavailable");
    D.bps = solver_blocks_per_sm();  // the same resident blocks per SM as a plan
    if (D.bps < 1) return nfail(ULP_ERR_CUDA, "ulp_pcg_noalloc: solver does not fit on an SM");
    D.base = p;
    D.plan.hmaps.resize(1);  // the only host allocation, once per device
    D.ready = true;
  }

  // Layout of the array for this grid.
  Plan& pl = D.plan;
  pl.device = dev;
  pl.nsm = D.nsm;
  pl.bps = D.bps;
  pl.nmaps = 1;
  pl.R = default_tile_rows(1, &H, &W, D.nsm * D.bps * kWarps);  // same tiles as ulp_pcg
  pl.bx_elem = D.nsm * 4;
  ulp_options_default(&pl.opt);
  MapDesc& M = pl.hmaps[0];
  M = MapDesc{};
  M.H = H;
  M.W = W;
  M.pitch = (int)pitch;
  M.nsx = M.pitch / kStrip;
  M.nsy = (H + pl.R - 1) / pl.R;
  M.tile_base = 0;
  M.ntiles = M.nsx * M.nsy;
  M.refresh = (int)std::floor(std::sqrt((double)H * (double)W));
  if (M.refresh < 1) M.refresh = 1;
  pl.ntiles = M.ntiles;
  char* p = static_cast<char*>(D.base);
  const size_t e64 = a256((size_t)H * pitch * sizeof(double));
  double** f64[kPlanes] = {&M.f.dx, &M.f.dy, &M.f.U, &M.f.V, &M.f.D, &M.f.Dinv, &M.f.b,
                           &M.f.phi, &M.f.phi_prev, &M.f.r, &M.f.s, &M.f.q, &M.f.d0, &M.f.d1};
  for (double** q : f64) { *q = reinterpret_cast<double*>(p); p += e64; }
  pl.dmaps = reinterpret_cast<MapDesc*>(p); p += a256(sizeof(MapDesc));
  pl.dstate = reinterpret_cast<MapState*>(p); p += a256(sizeof(MapState));
  pl.dstats = reinterpret_cast<MapStats*>(p); p += a256(sizeof(MapStats));
  pl.P0 = reinterpret_cast<double*>(p); p += a256(sizeof(double) * M.ntiles);
  pl.P1 = reinterpret_cast<double*>(p); p += a256(sizeof(double) * M.ntiles);
  pl.P2 = reinterpret_cast<double*>(p); p += a256(sizeof(double) * M.ntiles);
  pl.outer_part = reinterpret_cast<double*>(p); p += a256(sizeof(double) * 2 * pl.bx_elem);
  pl.bar = reinterpret_cast<Barrier*>(p); p += a256(sizeof(Barrier));
  pl.n_active = reinterpret_cast<int*>(p); p += a256(sizeof(int));
  const size_t used = (size_t)(p - static_cast<char*>(D.base));
  if (used > kNoAllocBytes) return nfail(ULP_ERR_INVALID, "ulp_pcg_noalloc: workspace layout exceeds the array");

  // Everything this call reads before writing starts at zero.
  if (cudaMemsetAsync(D.base, 0, used, st) != cudaSuccess) return nfail(ULP_ERR_CUDA, "ulp_pcg_noalloc: memset");
  k_store_map<<<1, 1, 0, st>>>(M, pl.dmaps);
  PcgArgs a{};
  a.maps = pl.dmaps;
  a.st = pl.dstate;
  a.nmaps = 1;
  a.ntiles = pl.ntiles;
  a.R = pl.R;
  a.P0 = pl.P0;
  a.P1 = pl.P1;
  a.P2 = pl.P2;
  a.bar = pl.bar;
  a.n_active = pl.n_active;
  a.stop_mode = ULP_STOP_RELRES;
  a.tol2 = tol * tol;
  a.lmax = max_inner;
  a.timeout_ns = (unsigned long long)(pl.opt.spin_timeout_s * 1e9);
  a.omega = 1.0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_begin(pl, st);
  if (e == cudaSuccess) e = launch_to_plane(pl, U, M.f.U, st);
  if (e == cudaSuccess) e = launch_to_plane(pl, V, M.f.V, st);
  if (e == cudaSuccess) e = launch_diag(pl, st);
  if (e == cudaSuccess) e = launch_to_plane(pl, b, M.f.b, st);
  if (e == cudaSuccess) e = launch_to_plane(pl, phi, M.f.phi, st);
  if (e == cudaSuccess) e = launch_pcg64(pl, precond, a, st, nullptr, nullptr);
  if (e == cudaSuccess) e = launch_outer_error(pl, 0.0, 1, st);
  if (e == cudaSuccess) e = launch_from_plane(pl, M.f.phi, phi, st);
  if (e != cudaSuccess) return nfail(ULP_ERR_CUDA, cudaGetErrorString(e));
  if (!stats) return ULP_OK;
  MapStats hs;
  if (cudaMemcpyAsync(&hs, pl.dstats, sizeof(MapStats), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return nfail(ULP_ERR_CUDA, "ulp_pcg_noalloc: reading statistics");
  std::memset(stats, 0, sizeof(*stats));
  stats->status = hs.status;
  stats->outer = hs.outer;
  stats->inner_total = hs.inner_total;
  for (int k = 0; k < ULP_MAX_OUTER_STATS; ++k) {
    stats->inner[k] = hs.inner[k];
    stats->relres[k] = hs.relres[k];
    stats->outer_err[k] = hs.outer_err[k];
  }
  // a solver error is recorded for ulp_last_error() with the same wording as ulp_pcg's
  if (hs.status < 0)
    return nfail(hs.status, hs.status == ULP_ERR_TIMEOUT     ? "an in-kernel wait ran out"
                            : hs.status == ULP_ERR_BREAKDOWN ? "PCG breakdown (d^T A d <= 0 or not finite)"
                                                             : "solver error");
  return hs.status;
}
