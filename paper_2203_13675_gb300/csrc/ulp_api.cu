// ulp_api.cu -- C ABI of the GB300 L^p phase-unwrapping library: plans
// (workspace ownership), argument checks, and the host orchestration of
// Algorithm 1 (outer reweighting passes around the persistent PCG engine).
// All control decisions of the iteration stay on the device, so a call
// enqueues a fixed sequence of kernels and never waits for the GPU unless
// statistics are requested.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>

#include "ulp_host.h"

using namespace ulp;

struct ulp_plan_s {
  Plan p;
};

static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// Records msg as the calling thread's last error (for files other than this one).
int ulp::set_error(int code, const char* msg) { return fail(code, "%s", msg); }

#define ULP_CU(x)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (x);                                                           \
    if (e_ != cudaSuccess) return fail(ULP_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

extern "C" void ulp_options_default(ulp_options* o) {
  std::memset(o, 0, sizeof(*o));
  o->stop_mode = ULP_STOP_RELRES;
  o->outer_tol = 1e-6;
  o->refresh = 0;
  o->omega = 1.0;
  o->precision = ULP_PRECISION_FP64;
  o->phi0_mode = ULP_PHI0_ZERO;
  o->tile_rows = 0;
  o->blocks_per_sm = 0;
  o->spin_timeout_s = 2.0;
}

extern "C" const char* ulp_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ plans
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static void destroy_plan(Plan& pl) {
  for (ulp_plan s : pl.sub) ulp_plan_destroy(s);
  pl.sub.clear();
  for (cudaStream_t s : pl.sub_st) cudaStreamDestroy(s);
  pl.sub_st.clear();
  for (cudaEvent_t e : pl.sub_ev) cudaEventDestroy(e);
  pl.sub_ev.clear();
  destroy_fcg(pl);
  if (pl.dct) dct_destroy(pl.dct);
  if (pl.dct_mem) cudaFree(pl.dct_mem);
  pl.dct = nullptr;
  pl.dct_mem = nullptr;
  if (pl.mg) mg_destroy(pl.mg);
  if (pl.mg_mem) cudaFree(pl.mg_mem);
  pl.mg = nullptr;
  pl.mg_mem = nullptr;
  if (pl.graph_exec) cudaGraphExecDestroy(pl.graph_exec);
  if (pl.cap_stream) cudaStreamDestroy(pl.cap_stream);
  pl.graph_exec = nullptr;
  pl.cap_stream = nullptr;
  for (cudaEvent_t e : pl.ev_pool) cudaEventDestroy(e);
  pl.ev_pool.clear();
  for (cudaEvent_t e : pl.ph_pool) cudaEventDestroy(e);
  pl.ph_pool.clear();
  if (pl.arena) cudaFree(pl.arena);
  pl.arena = nullptr;
}

// Next (start, stop) event pair for timing one solver launch, or nulls when
// profiling is off.
static void next_events(Plan& pl, cudaEvent_t* e0, cudaEvent_t* e1) {
  *e0 = *e1 = nullptr;
  if (!pl.opt.profile) return;
  while (pl.ev_pool.size() < pl.ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    pl.ev_pool.push_back(e);
  }
  *e0 = pl.ev_pool[pl.ev_used];
  *e1 = pl.ev_pool[pl.ev_used + 1];
  pl.ev_used += 2;
}

void ulp::phase_mark(Plan& pl, cudaStream_t st, int tag) {
  if (pl.ph_pool.size() < pl.ph_used + 1) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    pl.ph_pool.push_back(e);
    pl.ph_tag.push_back(-1);
  }
  pl.ph_tag[pl.ph_used] = tag;
  cudaEventRecord(pl.ph_pool[pl.ph_used], st);
  pl.ph_used += 1;
}

// Rows per warp tile: about one tile per resident warp of the persistent
// solver (static round-robin assignment, so equal counts balance the work),
// between 4 and 64 rows so the two halo rows stay amortised.
int ulp::solver_blocks_per_sm() {
  int occ = 1 << 30;
  for (int kind : {kIdentity, kJacobi}) {
    const int o = pcg64_max_blocks_per_sm(kind), o2 = pcg32_max_blocks_per_sm(kind);
    occ = o < occ ? o : occ;
    occ = o2 < occ ? o2 : occ;
  }
  return occ;
}

int ulp::sweep_blocks_per_sm() {
  const int a = pcg64_max_blocks_per_sm(kIlu), b = pcg64_max_blocks_per_sm(kSsor);
  return a < b ? a : b;
}

int ulp::default_tile_rows(int n, const int* H, const int* W, int resident_warps) {
  double cells = 0.0;  // rows x 64-column strips over all maps
  for (int m = 0; m < n; ++m) cells += (double)H[m] * ((W[m] + kStrip - 1) / kStrip);
  int R = (int)std::ceil(cells / (resident_warps > 0 ? resident_warps : 1));
  return R < 4 ? 4 : (R > 64 ? 64 : R);
}

static int plan_init(Plan& pl, int n, const int* H, const int* W, const ulp_options* opt) {
  if (n < 1 || n > kMaxMaps) return fail(ULP_ERR_INVALID, "map count %d outside [1, %d]", n, kMaxMaps);
  for (int m = 0; m < n; ++m) {
    if (H[m] < 2 || W[m] < 2) return fail(ULP_ERR_INVALID, "map %d: H=%d W=%d (need >= 2)", m, H[m], W[m]);
    if ((long long)H[m] * W[m] > (1LL << 31)) return fail(ULP_ERR_INVALID, "map %d too large", m);
  }
  if (opt) pl.opt = *opt; else ulp_options_default(&pl.opt);
  if (!(pl.opt.spin_timeout_s > 0.0)) pl.opt.spin_timeout_s = 2.0;
  if (!(pl.opt.omega > 0.0 && pl.opt.omega < 2.0)) return fail(ULP_ERR_INVALID, "omega must be in (0, 2)");
  if (pl.opt.precision != ULP_PRECISION_FP64 && pl.opt.precision != ULP_PRECISION_MIXED)
    return fail(ULP_ERR_INVALID, "unknown precision %d", pl.opt.precision);
  ULP_CU(cudaGetDevice(&pl.device));
  ULP_CU(cudaDeviceGetAttribute(&pl.nsm, cudaDevAttrMultiProcessorCount, pl.device));
  int coop = 0;
  ULP_CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, pl.device));
  if (!coop) return fail(ULP_ERR_UNSUPPORTED, "device lacks cooperative launch");
  pl.nmaps = n;
  const int occ = solver_blocks_per_sm();
  if (occ < 1 || sweep_blocks_per_sm() < 1) return fail(ULP_ERR_CUDA, "persistent solver does not fit on an SM");
  pl.bps = pl.opt.blocks_per_sm > 0 && pl.opt.blocks_per_sm < occ ? pl.opt.blocks_per_sm : occ;
  pl.bps_sweep = sweep_blocks_per_sm() < pl.bps ? sweep_blocks_per_sm() : pl.bps;
  pl.R = pl.opt.tile_rows > 0 ? pl.opt.tile_rows : default_tile_rows(n, H, W, pl.nsm * pl.bps * kWarps);

  // geometry and arena layout
  pl.hmaps.assign(n, MapDesc{});
  size_t bytes = 0;
  int tiles = 0, bands = 0;
  std::vector<size_t> plane_off(n);
  for (int m = 0; m < n; ++m) {
    MapDesc& M = pl.hmaps[m];
    M.H = H[m];
    M.W = W[m];
    M.pitch = (W[m] + kStrip - 1) / kStrip * kStrip;
    M.nsx = M.pitch / kStrip;
    M.nsy = (H[m] + pl.R - 1) / pl.R;
    M.tile_base = tiles;
    M.ntiles = M.nsx * M.nsy;
    tiles += M.ntiles;
    M.nbands = (H[m] + 31) / 32;
    M.band_base = bands;
    bands += M.nbands;
    long long rf = pl.opt.refresh > 0 ? pl.opt.refresh
                                      : (long long)std::floor(std::sqrt((double)H[m] * (double)W[m]));
    if (pl.opt.refresh <= 0 && pl.opt.precision == ULP_PRECISION_MIXED) rf = 20;
    if (rf < 1) rf = 1;
    if (rf > (1LL << 30)) rf = 1LL << 30;
    M.refresh = (int)rf;
    plane_off[m] = bytes;
    const size_t e = (size_t)M.H * M.pitch;
    bytes += 20 * align256(e * sizeof(double));   // FP64 planes
    bytes += 13 * align256(e * sizeof(float));    // FP32 planes
    bytes += align256(e);                         // mask
    bytes += 2 * align256((size_t)M.nbands * M.pitch * sizeof(double));  // sweep exchange rows
  }
  pl.ntiles = tiles;
  pl.nbands = bands;
  pl.bx_elem = pl.nsm * 4;
  const size_t off_maps = bytes;
  bytes += align256(sizeof(MapDesc) * n);
  const size_t off_state = bytes;
  bytes += align256(sizeof(MapState) * n);
  const size_t off_stats = bytes;
  bytes += align256(sizeof(MapStats) * n);
  const size_t off_part = bytes;
  bytes += 3 * align256(sizeof(double) * tiles);
  const size_t off_outer = bytes;
  bytes += align256(sizeof(double) * 2 * (size_t)n * pl.bx_elem);
  const size_t off_bar = bytes;
  bytes += align256(sizeof(Barrier)) + align256(sizeof(int));
  const size_t off_pt = bytes;
  bytes += 2 * align256(sizeof(double) * n);
  const size_t off_args = bytes;
  bytes += align256(sizeof(PcgArgs));

  cudaError_t e = cudaMalloc(&pl.arena, bytes);
  if (e != cudaSuccess) {
    pl.arena = nullptr;
    cudaGetLastError();
    return fail(ULP_ERR_NOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  pl.arena_bytes = bytes;
  ULP_CU(cudaMemset(pl.arena, 0, bytes));
  char* base = static_cast<char*>(pl.arena);
  for (int m = 0; m < n; ++m) {
    MapDesc& M = pl.hmaps[m];
    const size_t e64 = align256((size_t)M.H * M.pitch * sizeof(double));
    const size_t e32 = align256((size_t)M.H * M.pitch * sizeof(float));
    char* p = base + plane_off[m];
    double** f64[] = {&M.f.dx, &M.f.dy, &M.f.U, &M.f.V, &M.f.D, &M.f.Dinv, &M.f.b, &M.f.phi,
                      &M.f.phi_prev, &M.f.r, &M.f.s, &M.f.q, &M.f.d0, &M.f.d1, &M.f.piv, &M.f.y,
                      &M.f.cw, &M.f.cn, &M.f.ce, &M.f.cs};
    for (double** q : f64) { *q = reinterpret_cast<double*>(p); p += e64; }
    float** f32[] = {&M.h.U, &M.h.V, &M.h.Dinv, &M.h.x, &M.h.r, &M.h.s, &M.h.q,
                     &M.h.d0, &M.h.d1, &M.h.cw, &M.h.cn, &M.h.pinv, &M.h.y};
    for (float** q : f32) { *q = reinterpret_cast<float*>(p); p += e32; }
    M.f.mask = reinterpret_cast<uint8_t*>(p);
    p += align256((size_t)M.H * M.pitch);
    M.xf = reinterpret_cast<double*>(p);
    p += align256((size_t)M.nbands * M.pitch * sizeof(double));
    M.xb = reinterpret_cast<double*>(p);
  }
  pl.dmaps = reinterpret_cast<MapDesc*>(base + off_maps);
  pl.dstate = reinterpret_cast<MapState*>(base + off_state);
  pl.dstats = reinterpret_cast<MapStats*>(base + off_stats);
  pl.P0 = reinterpret_cast<double*>(base + off_part);
  pl.P1 = reinterpret_cast<double*>(base + off_part + align256(sizeof(double) * tiles));
  pl.P2 = reinterpret_cast<double*>(base + off_part + 2 * align256(sizeof(double) * tiles));
  pl.outer_part = reinterpret_cast<double*>(base + off_outer);
  pl.bar = reinterpret_cast<Barrier*>(base + off_bar);
  pl.n_active = reinterpret_cast<int*>(base + off_bar + align256(sizeof(Barrier)));
  pl.d_p = reinterpret_cast<double*>(base + off_pt);
  pl.d_tau = reinterpret_cast<double*>(base + off_pt + align256(sizeof(double) * n));
  pl.dargs = reinterpret_cast<PcgArgs*>(base + off_args);
  ULP_CU(cudaMemcpy(pl.dmaps, pl.hmaps.data(), sizeof(MapDesc) * n, cudaMemcpyHostToDevice));
  if (n == 1) {  // DCT preconditioner matrices and buffers (single-map plans)
    e = cudaMalloc(&pl.dct_mem, dct_bytes(H[0], W[0]));
    if (e != cudaSuccess) {
      pl.dct_mem = nullptr;
      cudaGetLastError();
      return fail(ULP_ERR_NOMEM, "cudaMalloc(DCT buffers): %s", cudaGetErrorString(e));
    }
    pl.dct = dct_create(H[0], W[0], pl.dct_mem);
    if (!pl.dct) return fail(ULP_ERR_CUDA, "DCT preconditioner set-up failed");
    e = cudaMalloc(&pl.mg_mem, mg_bytes(H[0], W[0]));
    if (e != cudaSuccess) {
      pl.mg_mem = nullptr;
      cudaGetLastError();
      return fail(ULP_ERR_NOMEM, "cudaMalloc(multigrid levels): %s", cudaGetErrorString(e));
    }
    pl.mg = mg_create(pl.hmaps[0], pl.mg_mem, pl.nsm, pl.ntiles);
  }
  ULP_CU(cudaDeviceSynchronize());  // workspace zeroed before any stream may use it
  return ULP_OK;
}

extern "C" int ulp_plan_create_batched(int n, const int* H, const int* W, const ulp_options* opt,
                                       ulp_plan* out) {
  if (!out || !H || !W) return fail(ULP_ERR_INVALID, "null argument");
  *out = nullptr;
  ulp_plan_s* p = new ulp_plan_s();
  int rc = plan_init(p->p, n, H, W, opt);
  if (rc != ULP_OK) {
    destroy_plan(p->p);
    delete p;
    return rc;
  }
  *out = p;
  return ULP_OK;
}

extern "C" int ulp_plan_create(int H, int W, const ulp_options* opt, ulp_plan* out) {
  return ulp_plan_create_batched(1, &H, &W, opt, out);
}

extern "C" void ulp_plan_destroy(ulp_plan plan) {
  if (!plan) return;
  destroy_plan(plan->p);
  delete plan;
}

// ------------------------------------------------------------------ solve
struct PT {
  double p[64];
  double tau[64];
};
__global__ void k_set_pt(PT pt, double* p, double* tau, int first, int n) {
  const int t = threadIdx.x;
  if (t < n) {
    p[first + t] = pt.p[t];
    tau[first + t] = pt.tau[t];
  }
}

// preconditioners that run in the graph-driven flexible CG (single-map plans)
static bool is_fcg_kind(int precond) {
  return precond == ULP_PRECOND_DCT || precond == ULP_PRECOND_LEARNED || precond == ULP_PRECOND_MG ||
         precond == ULP_PRECOND_RBSSOR || precond == ULP_PRECOND_RBILU;
}

static int check_solver_args(int precond, double tol, int max_outer) {
  if (precond < ULP_PRECOND_IDENTITY || precond > ULP_PRECOND_RBILU)
    return fail(ULP_ERR_INVALID, "unknown preconditioner %d", precond);

  if (!(tol > 0.0)) return fail(ULP_ERR_INVALID, "tol must be > 0");
  if (max_outer < 1) return fail(ULP_ERR_INVALID, "max_outer must be >= 1");
  return ULP_OK;
}

static void fill_stats(const MapStats& d, ulp_stats* s) {
  std::memset(s, 0, sizeof(*s));
  s->status = d.status;
  s->outer = d.outer;
  s->inner_total = d.inner_total;
  for (int k = 0; k < ULP_MAX_OUTER_STATS; ++k) {
    s->inner[k] = d.inner[k];
    s->relres[k] = d.relres[k];
    s->outer_err[k] = d.outer_err[k];
  }
  s->fallbacks = d.fallbacks;
  s->setup_ms = 1e-6 * (double)d.setup_ns;
}

static PcgArgs pcg_args(const Plan& pl, double tol, int max_inner) {
  PcgArgs a{};
  a.maps = pl.dmaps;
  a.st = pl.dstate;
  a.nmaps = pl.nmaps;
  a.ntiles = pl.ntiles;
  a.nbands = pl.nbands;
  a.R = pl.R;
  a.P0 = pl.P0;
  a.P1 = pl.P1;
  a.P2 = pl.P2;
  a.bar = pl.bar;
  a.n_active = pl.n_active;
  a.stop_mode = pl.opt.stop_mode;
  a.tol2 = tol * tol;
  a.lmax = max_inner;
  a.timeout_ns = (unsigned long long)(pl.opt.spin_timeout_s * 1e9);
  a.omega = pl.opt.omega;
  a.stall_window = pl.opt.stall_window > 0 ? pl.opt.stall_window : 200;
  a.stats = pl.dstats;
  return a;
}

static int collect(Plan& pl, cudaStream_t st, ulp_stats* per_map) {
  std::vector<MapStats> hs(pl.nmaps);
  ULP_CU(cudaMemcpyAsync(hs.data(), pl.dstats, sizeof(MapStats) * pl.nmaps, cudaMemcpyDeviceToHost, st));
  ULP_CU(cudaStreamSynchronize(st));
  int worst = ULP_OK;
  for (int m = 0; m < pl.nmaps; ++m) {
    if (per_map) fill_stats(hs[m], per_map + m);
    const int s = hs[m].status;
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
    else if (s == ULP_WARN_MAXITER && worst == ULP_OK) worst = s;
  }
  pl.last_status = worst;
  if (worst < 0) {
    const char* why = worst == ULP_ERR_TIMEOUT   ? "an in-kernel wait ran out"
                      : worst == ULP_ERR_BREAKDOWN ? "PCG breakdown (d^T A d <= 0 or not finite)"
                      : worst == ULP_ERR_INVALID   ? "non-finite wrapped phase"
                                                   : "solver error";
    fail(worst, "%s", why);
  }
  return worst;
}

// Outer passes enqueued before the host first looks at whether any map is still in its
// outer loop (calls with more passes than this; see enqueue_call).
constexpr int kOuterAhead = 8;

// 1 if any map of the plan is still in its outer loop: the maps' flags read after the
// work enqueued so far (the call waits for it).
static int any_outer_active(Plan& pl, cudaStream_t st) {
  std::vector<int> act(pl.nmaps, 0);
  if (cudaMemcpy2DAsync(act.data(), sizeof(int), &pl.dstate[0].outer_active, sizeof(MapState), sizeof(int),
                        pl.nmaps, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return -1;
  for (int v : act)
    if (v) return 1;
  return 0;
}

// Enqueues one call of Algorithm 1 for every map of the plan on stream st.  The passes
// decide on the device whether they run; a pass after the outer loop has stopped returns
// at once, but its launches still cost tens of microseconds.  So with more than
// kOuterAhead passes, and when the call may wait (not under stream capture, not a plan
// whose calls run beside others), the host stops enqueuing passes once every map has left
// its outer loop, looking after every kOuterAhead passes.
static int enqueue_call(Plan& pl, const ulp_map* maps, int precond, double tol, int max_outer, int max_inner,
                        cudaStream_t st, bool mixed, bool may_wait) {
  for (int first = 0; first < pl.nmaps; first += 64) {
    PT pt{};
    const int cnt = pl.nmaps - first < 64 ? pl.nmaps - first : 64;
    for (int t = 0; t < cnt; ++t) {
      pt.p[t] = maps[first + t].p;
      pt.tau[t] = maps[first + t].eps;
    }
    pl.kernel_launches += 1;
    k_set_pt<<<1, 64, 0, st>>>(pt, pl.d_p, pl.d_tau, first, cnt);
  }
  ULP_CU(cudaGetLastError());
  ULP_CU(launch_begin(pl, st));
  const bool user_phi0 = pl.opt.phi0_mode == ULP_PHI0_USER;
  for (int m = 0; m < pl.nmaps; ++m)
    ULP_CU(launch_pack(pl, m, maps[m].psi, maps[m].mask, user_phi0 ? maps[m].phi : nullptr, st));
  ULP_CU(launch_check(pl, st));
  const PcgArgs a = pcg_args(pl, tol, max_inner);
  // the mixed multigrid form takes its weights in FP32 straight into the planes it reads
  pl.system_x = mixed && precond == ULP_PRECOND_MG && pl.nmaps == 1;
  for (int k = 0; k < max_outer; ++k) {
    if (pl.system_x) ULP_CU(launch_system_x(pl, pl.d_p, pl.d_tau, st));
    else ULP_CU(launch_system(pl, pl.d_p, pl.d_tau, st));
    cudaEvent_t e0, e1;
    next_events(pl, &e0, &e1);
    if (is_fcg_kind(precond)) ULP_CU(launch_fcg(pl, precond, a, st, e0, e1));
    else if (mixed) ULP_CU(launch_pcg32(pl, precond, a, st, e0, e1));
    else ULP_CU(launch_pcg64(pl, precond, a, st, e0, e1));
    ULP_CU(launch_outer_error(pl, pl.opt.outer_tol, max_outer, st));
    if (may_wait && !pl.concurrent && max_outer > kOuterAhead && (k + 1) % kOuterAhead == 0 && k + 1 < max_outer) {
      const int act = any_outer_active(pl, st);
      if (act < 0) return fail(ULP_ERR_CUDA, "reading the outer-loop flags: %s", cudaGetErrorString(cudaGetLastError()));
      if (act == 0) break;
    }
  }
  for (int m = 0; m < pl.nmaps; ++m) ULP_CU(launch_unpack(pl, m, maps[m].phi, st));
  return ULP_OK;
}

// Replays the plan's captured call when the arguments are the ones it was
// captured with, capturing it (on the plan's own stream) otherwise.
static int graph_call(Plan& pl, const ulp_map* maps, int precond, double tol, int max_outer, int max_inner,
                      cudaStream_t st, bool mixed) {
  std::vector<unsigned char> key(sizeof(ulp_map) * pl.nmaps + sizeof(int) * 3 + sizeof(double));
  unsigned char* k = key.data();
  std::memcpy(k, maps, sizeof(ulp_map) * pl.nmaps);
  k += sizeof(ulp_map) * pl.nmaps;
  const int ints[3] = {precond, max_outer, max_inner};
  std::memcpy(k, ints, sizeof(ints));
  std::memcpy(k + sizeof(ints), &tol, sizeof(double));
  if (!pl.graph_exec || key != pl.graph_key) {
    if (pl.graph_exec) {
      cudaGraphExecDestroy(pl.graph_exec);
      pl.graph_exec = nullptr;
    }
    if (!pl.cap_stream) ULP_CU(cudaStreamCreateWithFlags(&pl.cap_stream, cudaStreamNonBlocking));
    const long long before = pl.kernel_launches;
    ULP_CU(cudaStreamBeginCapture(pl.cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_call(pl, maps, precond, tol, max_outer, max_inner, pl.cap_stream, mixed, false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(pl.cap_stream, &g);
    if (rc != ULP_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(ULP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&pl.graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      pl.graph_exec = nullptr;
      return fail(ULP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    pl.graph_key = key;
    pl.graph_kernels = pl.kernel_launches - before;
    pl.kernel_launches = before;
  }
  ULP_CU(cudaGraphLaunch(pl.graph_exec, st));
  pl.kernel_launches += pl.graph_kernels;
  pl.solver_launches += max_outer;
  return ULP_OK;
}

// Multigrid on a batched plan: every map on a single-map plan of its own (made on the first
// such call, with the batch's options), the maps spread over a few streams forked from the
// caller's stream and joined back into it, largest first on the least-loaded stream.  Each
// map's call is exactly ulp_unwrap on its plan.
constexpr int kBatchStreams = 8;
static int batched_sub_call(Plan& pl, const ulp_map* maps, int precond, double tol, int max_outer, int max_inner,
                            cudaStream_t st, ulp_stats* per_map) {
  const int n = pl.nmaps;
  if (pl.sub.empty()) {
    std::vector<int> order(n);
    for (int m = 0; m < n; ++m) order[m] = m;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      return (long long)pl.hmaps[a].H * pl.hmaps[a].W > (long long)pl.hmaps[b].H * pl.hmaps[b].W;
    });
    const int ns = n < kBatchStreams ? n : kBatchStreams;
    std::vector<long long> load(ns, 0);
    pl.sub.assign(n, nullptr);
    pl.sub_stream.assign(n, 0);
    for (int m : order) {
      int best = 0;
      for (int s = 1; s < ns; ++s)
        if (load[s] < load[best]) best = s;
      pl.sub_stream[m] = best;
      load[best] += (long long)pl.hmaps[m].H * pl.hmaps[m].W;
    }
    ulp_options o = pl.opt;
    o.graph = 0;
    for (int m = 0; m < n; ++m) {
      const int rc = ulp_plan_create(pl.hmaps[m].H, pl.hmaps[m].W, &o, &pl.sub[m]);
      if (rc != ULP_OK) {
        for (ulp_plan s : pl.sub) ulp_plan_destroy(s);
        pl.sub.clear();
        return rc;
      }
      pl.sub[m]->p.concurrent = true;  // the maps' calls run side by side on several streams
    }
    ULP_CU(cudaSetDevice(pl.device));
    pl.sub_st.assign(ns, nullptr);
    for (int s = 0; s < ns; ++s) ULP_CU(cudaStreamCreateWithFlags(&pl.sub_st[s], cudaStreamNonBlocking));
    pl.sub_ev.assign(ns + 1, nullptr);
    for (int s = 0; s <= ns; ++s) ULP_CU(cudaEventCreateWithFlags(&pl.sub_ev[s], cudaEventDisableTiming));
  }
  const int ns = (int)pl.sub_st.size();
  long long host = 0;
  for (int m = 0; m < n; ++m) host -= pl.sub[m]->p.kernel_launches;
  ULP_CU(cudaEventRecord(pl.sub_ev[0], st));
  for (int s = 0; s < ns; ++s) ULP_CU(cudaStreamWaitEvent(pl.sub_st[s], pl.sub_ev[0], 0));
  for (int m = 0; m < n; ++m) {
    const int rc = ulp_unwrap_batched(pl.sub[m], maps + m, precond, tol, max_outer, max_inner,
                                      pl.sub_st[pl.sub_stream[m]], nullptr);
    if (rc != ULP_OK) return rc;
  }
  for (int s = 0; s < ns; ++s) {
    ULP_CU(cudaEventRecord(pl.sub_ev[1 + s], pl.sub_st[s]));
    ULP_CU(cudaStreamWaitEvent(st, pl.sub_ev[1 + s], 0));
  }
  pl.last_stream = st;
  // kernels of the call: the host launches on the maps' plans, and, where the statistics give
  // the inner iterations, the kernels their solve graphs ran (start + iterations x body per pass)
  for (int m = 0; m < n; ++m) host += pl.sub[m]->p.kernel_launches;
  pl.kernel_launches += host;
  if (!per_map) {
    pl.last_status = ULP_OK;
    return ULP_OK;
  }
  int worst = ULP_OK;
  for (int m = 0; m < n; ++m) {
    const int s = ulp_plan_last_status(pl.sub[m], per_map + m);
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
    else if (s == ULP_WARN_MAXITER && worst == ULP_OK) worst = s;
    const Plan& sp = pl.sub[m]->p;
    for (int k = 0; k < per_map[m].outer && k < ULP_MAX_OUTER_STATS; ++k)
      pl.kernel_launches += sp.fcg_start_kernels + per_map[m].inner[k] * sp.fcg_body_kernels;
  }
  pl.last_status = worst;
  return worst;
}

extern "C" int ulp_unwrap_batched(ulp_plan plan, const ulp_map* maps, int precond, double tol,
                                  int max_outer, int max_inner, void* cuda_stream, ulp_stats* per_map) {
  if (!plan || !maps) return fail(ULP_ERR_INVALID, "null argument");
  Plan& pl = plan->p;
  int rc = check_solver_args(precond, tol, max_outer);
  if (rc != ULP_OK) return rc;
  const bool mixed = pl.opt.precision == ULP_PRECISION_MIXED;
  if (mixed && precond != ULP_PRECOND_IDENTITY && precond != ULP_PRECOND_JACOBI && precond != ULP_PRECOND_MG)
    return fail(ULP_ERR_UNSUPPORTED, "mixed precision supports the identity, Jacobi and multigrid preconditioners");
  if (precond == ULP_PRECOND_DCT && (pl.nmaps != 1 || !pl.dct))
    return fail(ULP_ERR_UNSUPPORTED, "the DCT preconditioner is available on single-map plans");
  if (precond == ULP_PRECOND_MG && pl.nmaps == 1 && !pl.mg)
    return fail(ULP_ERR_UNSUPPORTED, "the multigrid preconditioner is not set up on this plan");
  if ((precond == ULP_PRECOND_RBSSOR || precond == ULP_PRECOND_RBILU) && pl.nmaps != 1)
    return fail(ULP_ERR_UNSUPPORTED, "the red-black preconditioners are available on single-map plans");
  if (precond == ULP_PRECOND_LEARNED && (pl.nmaps != 1 || !pl.unet))
    return fail(ULP_ERR_UNSUPPORTED, "the learned preconditioner needs a single-map plan and ulp_plan_set_unet");
  for (int m = 0; m < pl.nmaps; ++m) {
    if (!maps[m].psi || !maps[m].phi) return fail(ULP_ERR_INVALID, "map %d: null psi or phi", m);
    if (!(maps[m].p >= 0.0 && maps[m].p <= 2.0)) return fail(ULP_ERR_INVALID, "map %d: p outside [0, 2]", m);
    if (!(maps[m].eps > 0.0) || !std::isfinite(maps[m].eps)) return fail(ULP_ERR_INVALID, "map %d: eps must be > 0", m);
  }
  ULP_CU(cudaSetDevice(pl.device));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (precond == ULP_PRECOND_MG && pl.nmaps > 1)
    return batched_sub_call(pl, maps, precond, tol, max_outer, max_inner, st, per_map);
  pl.last_stream = st;
  // the DCT, learned and multigrid solves are themselves graphs with a WHILE node, which cannot be
  // nested: they run eagerly
  if (pl.opt.graph && !pl.opt.profile && !is_fcg_kind(precond))
    rc = graph_call(pl, maps, precond, tol, max_outer, max_inner, st, mixed);
  else rc = enqueue_call(pl, maps, precond, tol, max_outer, max_inner, st, mixed, true);
  if (rc != ULP_OK) return rc;
  if (per_map) return collect(pl, st, per_map);
  pl.last_status = ULP_OK;
  return ULP_OK;
}

extern "C" int ulp_unwrap(ulp_plan plan, const double* psi, const uint8_t* mask, double p, double eps,
                          int precond, double tol, int max_outer, int max_inner, double* phi,
                          void* cuda_stream, ulp_stats* stats) {
  if (!plan) return fail(ULP_ERR_INVALID, "null plan");
  if (plan->p.nmaps != 1) return fail(ULP_ERR_INVALID, "batched plan: use ulp_unwrap_batched");
  ulp_map mp{psi, mask, phi, p, eps};
  return ulp_unwrap_batched(plan, &mp, precond, tol, max_outer, max_inner, cuda_stream, stats);
}

extern "C" int ulp_plan_counters(ulp_plan plan, int reset, ulp_counters* out) {
  if (!plan || !out) return fail(ULP_ERR_INVALID, "null argument");
  Plan& pl = plan->p;
  ULP_CU(cudaSetDevice(pl.device));
  out->kernel_launches = pl.kernel_launches;
  out->solver_launches = pl.solver_launches;
  out->solver_ms = 0.0;
  out->timed_launches = (long long)(pl.ev_used / 2);
  for (size_t k = 0; k + 1 < pl.ev_used; k += 2) {
    ULP_CU(cudaEventSynchronize(pl.ev_pool[k + 1]));
    float ms = 0.f;
    ULP_CU(cudaEventElapsedTime(&ms, pl.ev_pool[k], pl.ev_pool[k + 1]));
    out->solver_ms += ms;
  }
  for (int k = 0; k < 6; ++k) {
    out->phase_ms[k] = 0.0;
    out->phase_launches[k] = 0;
  }
  out->graph_start_kernels = pl.fcg_start_kernels;
  out->graph_body_kernels = pl.fcg_body_kernels;
  for (size_t k = 1; k < pl.ph_used; ++k) {
    const int t = pl.ph_tag[k];
    if (t < 0 || t > 5) continue;
    ULP_CU(cudaEventSynchronize(pl.ph_pool[k]));
    float ms = 0.f;
    ULP_CU(cudaEventElapsedTime(&ms, pl.ph_pool[k - 1], pl.ph_pool[k]));
    out->phase_ms[t] += ms;
    out->phase_launches[t] += 1;
  }
  if (reset) {
    pl.kernel_launches = 0;
    pl.solver_launches = 0;
    pl.ev_used = 0;
    pl.ph_used = 0;
  }
  return ULP_OK;
}

extern "C" int ulp_plan_set_unet(ulp_plan plan, ulp_unet net) {
  if (!plan) return fail(ULP_ERR_INVALID, "null plan");
  Plan& pl = plan->p;
  if (net && (pl.nmaps != 1 || pl.opt.precision != ULP_PRECISION_FP64))
    return fail(ULP_ERR_UNSUPPORTED, "the learned preconditioner needs a single-map FP64 plan");
  Unet* u = net ? ulp_unet_impl(net) : nullptr;
  if (u != pl.unet && pl.fcg_kind == ULP_PRECOND_LEARNED) {
    ULP_CU(cudaSetDevice(pl.device));
    destroy_fcg(pl);  // the captured solve refers to the old network's buffers
  }
  pl.unet = u;
  return ULP_OK;
}

extern "C" int ulp_plan_last_status(ulp_plan plan, ulp_stats* stats) {
  if (!plan) return fail(ULP_ERR_INVALID, "null plan");
  Plan& pl = plan->p;
  ULP_CU(cudaSetDevice(pl.device));
  if (!pl.sub.empty()) {  // a multigrid batch: the worst over the maps' own plans, the first map's stats
    int worst = ULP_OK;
    for (size_t m = 0; m < pl.sub.size(); ++m) {
      ulp_stats s;
      const int r = ulp_plan_last_status(pl.sub[m], &s);
      if (m == 0 && stats) *stats = s;
      if (r < 0 && (worst >= 0 || r < worst)) worst = r;
      else if (r == ULP_WARN_MAXITER && worst == ULP_OK) worst = r;
    }
    return worst;
  }
  std::vector<ulp_stats> all(pl.nmaps);  // collect() writes one record per map; the caller gets the first
  const int rc = collect(pl, pl.last_stream, all.data());
  if (stats) *stats = all[0];
  return rc;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" int unwrap_lp(const double* psi, int H, int W, double p, double eps, int precond, double tol,
                         int max_outer, int max_inner, double* phi) {
  if (!psi || !phi) return fail(ULP_ERR_INVALID, "null psi or phi");
  if (H < 2 || W < 2) return fail(ULP_ERR_INVALID, "H=%d W=%d (need >= 2)", H, W);
  ulp_options o;
  ulp_options_default(&o);
  o.outer_tol = 0.0;
  ulp_plan plan = nullptr;
  int rc = ulp_plan_create(H, W, &o, &plan);
  if (rc != ULP_OK) return rc;
  const bool dev_in = is_device_ptr(psi), dev_out = is_device_ptr(phi);
  const size_t bytes = (size_t)H * W * sizeof(double);
  double *dpsi = const_cast<double*>(psi), *dphi = phi;
  if (!dev_in || !dev_out) {
    cudaError_t e = cudaSuccess;
    if (!dev_in) e = cudaMalloc(&dpsi, bytes);
    if (e == cudaSuccess && !dev_out) e = cudaMalloc(&dphi, bytes);
    if (e == cudaSuccess && !dev_in) e = cudaMemcpy(dpsi, psi, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      if (!dev_in && dpsi != psi) cudaFree(dpsi);
      if (!dev_out && dphi != phi) cudaFree(dphi);
      ulp_plan_destroy(plan);
      return fail(ULP_ERR_CUDA, "staging: %s", cudaGetErrorString(e));
    }
  }
  ulp_stats stats;
  rc = ulp_unwrap(plan, dpsi, nullptr, p, eps, precond, tol, max_outer, max_inner, dphi, nullptr, &stats);
  if (rc >= 0 && !dev_out) {
    cudaError_t e = cudaMemcpy(phi, dphi, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = fail(ULP_ERR_CUDA, "copy out: %s", cudaGetErrorString(e));
  }
  if (!dev_in) cudaFree(dpsi);
  if (!dev_out) cudaFree(dphi);
  ulp_plan_destroy(plan);
  return rc;
}

// ------------------------------------------------------------------ single steps
// Each builds a one-map workspace, runs the solver's own kernels, copies the
// result back to the caller's contiguous array and releases the workspace.
struct TempPlan {
  ulp_plan plan = nullptr;
  cudaStream_t st = nullptr;
  ~TempPlan() {
    if (plan) {
      cudaStreamSynchronize(st);
      ulp_plan_destroy(plan);
    }
  }
};

static int temp_plan(TempPlan& tp, int H, int W, const ulp_options* opt, void* stream) {
  tp.st = static_cast<cudaStream_t>(stream);
  return ulp_plan_create(H, W, opt, &tp.plan);
}

extern "C" int ulp_wrapped_diffs(const double* psi, int H, int W, double* dx, double* dy, void* stream) {
  if (!psi || !dx || !dy) return fail(ULP_ERR_INVALID, "null argument");
  TempPlan tp;
  int rc = temp_plan(tp, H, W, nullptr, stream);
  if (rc != ULP_OK) return rc;
  Plan& pl = tp.plan->p;
  ULP_CU(launch_begin(pl, tp.st));
  ULP_CU(launch_pack(pl, 0, psi, nullptr, nullptr, tp.st));
  ULP_CU(launch_from_plane(pl, pl.hmaps[0].f.dx, dx, tp.st));
  ULP_CU(launch_from_plane(pl, pl.hmaps[0].f.dy, dy, tp.st));
  ULP_CU(cudaStreamSynchronize(tp.st));
  return ULP_OK;
}

extern "C" int ulp_weights(const double* phi, const double* dx, const double* dy, const uint8_t* mask,
                           int H, int W, double p, double eps, double* U, double* V, double* b,
                           void* stream) {
  if (!phi || !dx || !dy || !U || !V) return fail(ULP_ERR_INVALID, "null argument");
  if (!(p >= 0.0 && p <= 2.0) || !(eps > 0.0)) return fail(ULP_ERR_INVALID, "p or eps out of range");
  TempPlan tp;
  int rc = temp_plan(tp, H, W, nullptr, stream);
  if (rc != ULP_OK) return rc;
  Plan& pl = tp.plan->p;
  const MapDesc& M = pl.hmaps[0];
  PT pt{};
  pt.p[0] = p;
  pt.tau[0] = eps;
  k_set_pt<<<1, 64, 0, tp.st>>>(pt, pl.d_p, pl.d_tau, 0, 1);
  ULP_CU(launch_begin(pl, tp.st));
  ULP_CU(launch_to_plane(pl, phi, M.f.phi, tp.st));
  ULP_CU(launch_to_plane(pl, dx, M.f.dx, tp.st));
  ULP_CU(launch_to_plane(pl, dy, M.f.dy, tp.st));
  ULP_CU(launch_mask_to_plane(pl, mask, tp.st));
  ULP_CU(launch_system(pl, pl.d_p, pl.d_tau, tp.st));
  ULP_CU(launch_from_plane(pl, M.f.U, U, tp.st));
  ULP_CU(launch_from_plane(pl, M.f.V, V, tp.st));
  if (b) ULP_CU(launch_from_plane(pl, M.f.b, b, tp.st));
  ULP_CU(cudaStreamSynchronize(tp.st));
  return ULP_OK;
}

// Loads caller weights U, V into a temporary plan and forms D, D^-1 (b = 0).
static int load_weights(Plan& pl, const double* U, const double* V, cudaStream_t st) {
  const MapDesc& M = pl.hmaps[0];
  ULP_CU(launch_begin(pl, st));
  ULP_CU(launch_to_plane(pl, U, M.f.U, st));
  ULP_CU(launch_to_plane(pl, V, M.f.V, st));
  ULP_CU(launch_diag(pl, st));
  return ULP_OK;
}

extern "C" int ulp_matvec(const double* U, const double* V, const double* x, int H, int W, double* y,
                          void* stream) {
  if (!U || !V || !x || !y) return fail(ULP_ERR_INVALID, "null argument");
  TempPlan tp;
  int rc = temp_plan(tp, H, W, nullptr, stream);
  if (rc != ULP_OK) return rc;
  Plan& pl = tp.plan->p;
  const MapDesc& M = pl.hmaps[0];
  rc = load_weights(pl, U, V, tp.st);
  if (rc != ULP_OK) return rc;
  ULP_CU(launch_to_plane(pl, x, M.f.r, tp.st));
  ULP_CU(launch_matvec(pl, M.f.r, M.f.q, tp.st));
  ULP_CU(launch_from_plane(pl, M.f.q, y, tp.st));
  ULP_CU(cudaStreamSynchronize(tp.st));
  return ULP_OK;
}

extern "C" int ulp_precond_apply(int precond, const double* U, const double* V, const uint8_t* mask,
                                 int H, int W, double omega, const double* r, double* s, void* stream) {
  if (!U || !V || !r || !s) return fail(ULP_ERR_INVALID, "null argument");
  int rc = check_solver_args(precond, 1.0, 1);
  if (rc != ULP_OK) return rc;
  ulp_options o;
  ulp_options_default(&o);
  o.omega = omega;
  TempPlan tp;
  rc = temp_plan(tp, H, W, &o, stream);
  if (rc != ULP_OK) return rc;
  Plan& pl = tp.plan->p;
  const MapDesc& M = pl.hmaps[0];
  rc = load_weights(pl, U, V, tp.st);
  if (rc != ULP_OK) return rc;
  if (precond == ULP_PRECOND_LEARNED) {
    return fail(ULP_ERR_UNSUPPORTED, "ulp_precond_apply: use ulp_unet_apply for the learned preconditioner");
  } else if (precond == ULP_PRECOND_IDENTITY || precond == ULP_PRECOND_JACOBI) {
    ULP_CU(launch_to_plane(pl, r, M.f.r, tp.st));
    ULP_CU(launch_jacobi_apply(pl, precond, M.f.r, M.f.s, tp.st));
  } else if (precond == ULP_PRECOND_RBSSOR || precond == ULP_PRECOND_RBILU) {
    ULP_CU(launch_to_plane(pl, r, M.f.r, tp.st));
    ULP_CU(rb_setup(pl, precond, nullptr, tp.st));
    ULP_CU(rb_apply(pl, precond, nullptr, tp.st));
  } else if (precond == ULP_PRECOND_MG) {
    ULP_CU(launch_to_plane(pl, r, M.f.r, tp.st));
    if (mask) ULP_CU(launch_mask_to_plane(pl, mask, tp.st));
    ULP_CU(mg_setup(*pl.mg, nullptr, tp.st));
    ULP_CU(mg_apply(*pl.mg, mask ? M.f.mask : nullptr, nullptr, tp.st));
  } else if (precond == ULP_PRECOND_DCT) {
    ULP_CU(launch_to_plane(pl, r, M.f.r, tp.st));
    if (mask) ULP_CU(launch_mask_to_plane(pl, mask, tp.st));
    ULP_CU(dct_apply(*pl.dct, M.f.r, M.pitch, mask ? M.f.mask : nullptr, M.f.s, tp.st));
    ULP_CU(cudaStreamSynchronize(tp.st));
    if (dct_error(*pl.dct)) return fail(ULP_ERR_TIMEOUT, "DCT GEMM wait ran out");
  } else {
    // the sweep solver's set-up and first s = M^-1 r, with b = r and phi = 0
    ULP_CU(launch_to_plane(pl, r, M.f.b, tp.st));
    PcgArgs a = pcg_args(pl, 1.0, 1);
    a.apply_only = 1;
    ULP_CU(launch_pcg64(pl, precond, a, tp.st, nullptr, nullptr));
  }
  ULP_CU(launch_from_plane(pl, M.f.s, s, tp.st));
  ULP_CU(cudaStreamSynchronize(tp.st));
  return ULP_OK;
}

namespace ulp {
// The inner PCG of ulp_pcg on an existing single-map plan of that size, with the plan's
// options (the training-pair harvest runs many solves on one plan).
int pcg_on_plan(ulp_plan plan, const double* U, const double* V, const double* b, int precond, double tol,
                int max_inner, double* phi, cudaStream_t st, ulp_stats* stats) {
  Plan& pl = plan->p;
  const MapDesc& M = pl.hmaps[0];
  int rc = load_weights(pl, U, V, st);
  if (rc != ULP_OK) return rc;
  ULP_CU(launch_to_plane(pl, b, M.f.b, st));
  ULP_CU(launch_to_plane(pl, phi, M.f.phi, st));
  if (precond == ULP_PRECOND_LEARNED) return fail(ULP_ERR_UNSUPPORTED, "ulp_pcg: the learned preconditioner needs a plan");
  if (is_fcg_kind(precond)) ULP_CU(launch_fcg(pl, precond, pcg_args(pl, tol, max_inner), st));
  else ULP_CU(launch_pcg64(pl, precond, pcg_args(pl, tol, max_inner), st, nullptr, nullptr));
  ULP_CU(launch_outer_error(pl, 0.0, 1, st));
  ULP_CU(launch_from_plane(pl, M.f.phi, phi, st));
  if (stats) return collect(pl, st, stats);
  ULP_CU(cudaStreamSynchronize(st));
  return ULP_OK;
}

// y = A(U, V) x on an existing single-map plan of that size.
int matvec_on_plan(ulp_plan plan, const double* U, const double* V, const double* x, double* y, cudaStream_t st) {
  Plan& pl = plan->p;
  const MapDesc& M = pl.hmaps[0];
  int rc = load_weights(pl, U, V, st);
  if (rc != ULP_OK) return rc;
  ULP_CU(launch_to_plane(pl, x, M.f.r, st));
  ULP_CU(launch_matvec(pl, M.f.r, M.f.q, st));
  ULP_CU(launch_from_plane(pl, M.f.q, y, st));
  return ULP_OK;
}
}  // namespace ulp

extern "C" int ulp_pcg(const double* U, const double* V, const double* b, int H, int W, int precond,
                       double tol, int max_inner, const ulp_options* opt, double* phi, void* stream,
                       ulp_stats* stats) {
  if (!U || !V || !b || !phi) return fail(ULP_ERR_INVALID, "null argument");
  int rc = check_solver_args(precond, tol, 1);
  if (rc != ULP_OK) return rc;
  TempPlan tp;
  rc = temp_plan(tp, H, W, opt, stream);
  if (rc != ULP_OK) return rc;
  return pcg_on_plan(tp.plan, U, V, b, precond, tol, max_inner, phi, tp.st, stats);
}
