// ulp_host.h -- host-side plan of the GB300 L^p phase-unwrapping library and
// the launchers each kernel file exports to the C ABI layer (internal).
#pragma once
#include <vector>

#include "../../include/unwrap_lp.h"
#include "ulp_internal.cuh"

namespace ulp {

struct DctPlan;  // ulp_dct.cu
struct Unet;     // ulp_unet.cu
struct MgPlan;   // ulp_mg.cu

struct Plan {
  int device = 0;
  int nsm = 0;
  int nmaps = 0;
  int ntiles = 0;
  int R = 32;                // rows per warp tile
  int bps = 1;               // resident blocks per SM of the persistent solvers
  int bx_elem = 1;           // blocks per map of the elementwise kernels
  bool system_x = false;     // the current call builds its system with launch_system_x
  bool concurrent = false;   // the plan's calls run beside others (a batched plan's per-map plans):
                             // a call never waits for the GPU
  ulp_options opt{};
  std::vector<MapDesc> hmaps;
  MapDesc* dmaps = nullptr;
  MapState* dstate = nullptr;
  MapStats* dstats = nullptr;
  double *P0 = nullptr, *P1 = nullptr, *P2 = nullptr;
  double* outer_part = nullptr;
  Barrier* bar = nullptr;
  int* n_active = nullptr;
  int nbands = 0;
  int bps_sweep = 1;         // resident blocks per SM of the sweep solvers
  DctPlan* dct = nullptr;    // DCT preconditioner buffers (single-map plans)
  void* dct_mem = nullptr;
  PcgArgs* dargs = nullptr;  // solver arguments in device memory (read by the graph-driven solve)
  cudaGraphExec_t fcg_exec = nullptr;       // flexible-CG solve graph (DCT preconditioner)
  unsigned long long fcg_cond = 0;          // its WHILE-node handle
  int fcg_kind = -1;                        // preconditioner the flexible-CG graph was built for
  long long fcg_start_kernels = 0;          // kernels of its start and of one WHILE-body execution
  long long fcg_body_kernels = 0;
  Unet* unet = nullptr;                     // learned preconditioner (not owned)
  MgPlan* mg = nullptr;                     // multigrid hierarchy (single-map plans)
  void* mg_mem = nullptr;
  long long fcg_gen = 0;                    // its workspace generation captured in fcg_exec
  double *d_p = nullptr, *d_tau = nullptr;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  cudaStream_t last_stream = nullptr;
  int last_status = 0;
  // instrumentation
  mutable long long kernel_launches = 0;
  mutable long long solver_launches = 0;
  std::vector<cudaEvent_t> ev_pool;      // pairs (start, stop) recorded around solver launches
  size_t ev_used = 0;
  // host-driven flexible CG (options.profile = 2): an event after every phase; ph_tag[k] is
  // the phase (0 A, 1 B, 2 R, 3 M, 4 D) of the interval that ends at event k, -1 for a start
  std::vector<cudaEvent_t> ph_pool;
  std::vector<int> ph_tag;
  size_t ph_used = 0;
  // multigrid batches: one single-map plan per map, run concurrently on a few streams (the
  // flexible-CG solve of each map is itself a graph with a WHILE node, which does not nest)
  std::vector<ulp_plan> sub;
  std::vector<int> sub_stream;              // stream index of each map
  std::vector<cudaStream_t> sub_st;
  std::vector<cudaEvent_t> sub_ev;          // fork event, then one join event per stream
  // captured call (options.graph): the executable graph, the arguments it was captured with
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned char> graph_key;
  long long graph_kernels = 0;
};

// ulp_api.cu: records msg as the calling thread's last error and returns code.
int set_error(int code, const char* msg);
// ulp_api.cu: rows per warp tile for n maps and the solver's resident warps.
int default_tile_rows(int n, const int* H, const int* W, int resident_warps);
// ulp_api.cu: resident blocks per SM that fix the tile geometry (FP64 and mixed
// Jacobi / identity solvers), and those of the sweep solvers.
int solver_blocks_per_sm();
int sweep_blocks_per_sm();

// ulp_fp64.cu
cudaError_t launch_pack(const Plan& pl, int m, const double* psi, const uint8_t* mask, const double* phi0,
                        cudaStream_t st);
cudaError_t launch_unpack(const Plan& pl, int m, double* phi, cudaStream_t st);
cudaError_t launch_begin(const Plan& pl, cudaStream_t st);
cudaError_t launch_check(const Plan& pl, cudaStream_t st);
cudaError_t launch_diag(const Plan& pl, cudaStream_t st);
cudaError_t launch_system(const Plan& pl, const double* d_p, const double* d_tau, cudaStream_t st);
// mixed multigrid form (single-map plans): FP32 weights and D^-1 in the map's FP32 planes, their
// FP64 promotions, D and b in the FP64 planes
cudaError_t launch_system_x(const Plan& pl, const double* d_p, const double* d_tau, cudaStream_t st);
cudaError_t launch_outer_error(const Plan& pl, double outer_tol, int max_outer, cudaStream_t st);
cudaError_t launch_pcg64(const Plan& pl, int kind, const PcgArgs& a, cudaStream_t st, cudaEvent_t e0 = nullptr,
                         cudaEvent_t e1 = nullptr);
int pcg64_max_blocks_per_sm(int kind);
void launch_pcg_reset(const Plan& pl, cudaStream_t st);

// ulp_dct.cu
size_t dct_bytes(int H, int W);
DctPlan* dct_create(int H, int W, void* mem);  // builds the matrices in mem (dct_bytes); null on failure
void dct_destroy(DctPlan* d);
// the split BF16 copy of r that the first GEMM reads: high plane returned, low plane in *lo
unsigned* dct_input(const DctPlan& d, int* ld_pairs, unsigned** lo);
// the mask's bit plane used by dct_apply(..., packed = true)
cudaError_t dct_prepare_mask(const DctPlan& d, const uint8_t* mask, int pitch, cudaStream_t st);
// packed: the BF16 copy of r (dct_input) and the mask bits (dct_prepare_mask) are
// already written, skip those passes
cudaError_t dct_apply(const DctPlan& d, const double* r, int pitch, const uint8_t* mask, double* s,
                      cudaStream_t st, bool packed = false);
int dct_error(const DctPlan& d);  // 1 if a GEMM wait ran out since the last call (clears the flag)

// ulp_fcg.cu
// ulp_mg.cu: aggregation multigrid on the map's planes (U, V, D^-1; r -> s, y as scratch)
size_t mg_bytes(int H, int W);
MgPlan* mg_create(const MapDesc& M, void* mem, int nsm, int ntiles);
void mg_destroy(MgPlan* p);
// coarse grids, once per solve; level0: make the map grid's FP32 weights and D^-1 from the FP64
// planes (false when launch_system_x already wrote them)
cudaError_t mg_setup(const MgPlan& p, const MapState* S, cudaStream_t st, bool level0 = true);
// packed: the FP32 copy of r (mg_input, the map's pitch) is already written; dots (device
// arguments of a flexible-CG solve, or null): the cycle's last kernel also does the solve's
// dot phase (r^T s, r^T r, beta, stop test), if mg_fuses_dots
// s32 (or null): s is written in FP32 there instead of the map's FP64 s plane (the mixed flexible CG)
// dots_init: the dot phase is the start of a solve (r^T s, r^T r, and b^T b from the
// per-tile partials that k_x_res left in P2)
// part: 0 the whole cycle; 1 all but its last kernel (the up step on the map's grid); 2 that
// last kernel alone (the host-driven replay times it on its own)
cudaError_t mg_apply(const MgPlan& p, const uint8_t* mask, const MapState* S, cudaStream_t st, bool packed = false,
                     const PcgArgs* dots = nullptr, float* s32 = nullptr, bool dots_init = false, int part = 0);
bool mg_fuses_dots(const MgPlan& p);
float* mg_input(const MgPlan& p);
int mg_levels(const MgPlan& p);

// ulp_rb.cu: red-black SSOR / ILU(0) on the map's planes (r -> s; ILU pivots in piv)
cudaError_t rb_setup(const Plan& pl, int kind, const MapState* S, cudaStream_t st);  // once per solve
cudaError_t rb_apply(const Plan& pl, int kind, const MapState* S, cudaStream_t st);

// ulp_unet.cu: workspace for B images of Hn x Wn (multiples of 128); 0, -5 (no memory) or -2
int unet_prepare(Unet& u, int B, int Hn, int Wn);
// s = rho N(r / rho, U, V) on one map; every kernel returns at once while *skip != 0
cudaError_t unet_apply_plane(Unet& u, const double* r, const double* U, const double* V, const uint8_t* mask, int H,
                             int W, int pitch, double* s, const int* skip, cudaStream_t st);
int unet_error(Unet& u);  // 1 if a tensor-core wait ran out since the last call (clears the flag)
long long unet_ws_gen(const Unet& u);  // changes whenever the workspace is reallocated
}  // namespace ulp
ulp::Unet* ulp_unet_impl(ulp_unet net);  // the network behind a C handle
namespace ulp {

// ulp_api.cu: records the event that ends a phase interval of the host-driven flexible CG
void phase_mark(Plan& pl, cudaStream_t st, int tag);

// ulp_api.cu: the inner PCG of ulp_pcg and the matvec of ulp_matvec on an existing single-map
// plan of that size (no allocation; the plan's options)
int pcg_on_plan(ulp_plan plan, const double* U, const double* V, const double* b, int precond, double tol,
                int max_inner, double* phi, cudaStream_t st, ulp_stats* stats);
int matvec_on_plan(ulp_plan plan, const double* U, const double* V, const double* x, double* y, cudaStream_t st);

// ulp_fcg.cu: the flexible-CG solve with the DCT, multigrid or learned preconditioner
cudaError_t launch_fcg(Plan& pl, int kind, const PcgArgs& a, cudaStream_t st, cudaEvent_t e0 = nullptr,
                       cudaEvent_t e1 = nullptr);
void destroy_fcg(Plan& pl);

// ulp_mixed.cu
cudaError_t launch_pcg32(const Plan& pl, int kind, const PcgArgs& a, cudaStream_t st, cudaEvent_t e0 = nullptr,
                         cudaEvent_t e1 = nullptr);
int pcg32_max_blocks_per_sm(int kind);
cudaError_t launch_matvec(const Plan& pl, const double* x, double* y, cudaStream_t st);
cudaError_t launch_jacobi_apply(const Plan& pl, int kind, const double* r, double* s, cudaStream_t st);
cudaError_t launch_to_plane(const Plan& pl, const double* src, double* dst, cudaStream_t st);
cudaError_t launch_from_plane(const Plan& pl, const double* src, double* dst, cudaStream_t st);
cudaError_t launch_mask_to_plane(const Plan& pl, const uint8_t* mask, cudaStream_t st);

}  // namespace ulp
