// Declarations shared by the host C ABI (nlinv.cu) and the per-grid-size
// kernel units (grid.cu, compiled once per FFT split G = G1 x G2): the plan,
// the frame/batch launch arguments, error handling, and the table of
// per-grid-size operations the host dispatches through.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "cluster.cuh"
#include "nlinv.h"
#include "phases.cuh"

namespace nlinv {

// ------------------------------------------------------------ errors
// Record a failed CUDA call (thread-local message) and map it to a code.
int cuda_fail(cudaError_t e, const char* what);

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return ::nlinv::cuda_fail(e_, #call); \
  } while (0)

#define CKL(what)                                           \
  do {                                                      \
    cudaError_t e_ = cudaGetLastError();                    \
    if (e_ != cudaSuccess) return ::nlinv::cuda_fail(e_, what); \
  } while (0)

#define RC(x)                        \
  do {                               \
    int rc_ = (x);                   \
    if (rc_ != NLINV_OK) return rc_; \
  } while (0)

constexpr int kMaxNewton = 32;
constexpr int kMaxBatch = 64;

// per-frame inputs and outputs
struct FrameIO {
  const float2* Y;
  const float* P;
  const float2* xprev;
  float2* xout;
  float2* rho_out;
  float2* img_out;
  const float2* xlast;    // regulariser of the last Newton step (x ref = damping * xlast), or null
  const unsigned* wait;   // before the last Newton step: wait until *wait != 0, or null
  unsigned* done;         // set to 1 once xout is written, or null
};

// barrier counter and completion flag of the frame group f of a launch, one
// 128-byte line each so that groups do not contend
constexpr int kBarStride = 32;   // unsigned words per frame group

struct FrameArgs {
  FrameIO io;
  int M, K;
  float damping;
  float alpha[kMaxNewton];
};

struct BatchArgs {
  int nf, M, K;
  float damping;
  float alpha[kMaxNewton];
  size_t fstride;             // bytes between the frames' workspaces
  FrameIO io[kMaxBatch];
};

// the workspace of frame f: every per-frame buffer moved by `off` bytes
__host__ __device__ __forceinline__ Ctx frame_ctx(Ctx C, size_t off) {
#define NLINV_ADV(T, p) C.p = (T*)((char*)C.p + off)
  NLINV_ADV(float2, c);
  NLINV_ADV(float2, h);
  NLINV_ADV(float2, v);
  NLINV_ADV(float2, s);
  NLINV_ADV(float2, kb);
  NLINV_ADV(float2, xn);
  NLINV_ADV(float2, xref);
  NLINV_ADV(float2, xcg);
  NLINV_ADV(float2, rb[0]);
  NLINV_ADV(float2, rb[1]);
  NLINV_ADV(float2, q);
  NLINV_ADV(float2, pb[0]);
  NLINV_ADV(float2, pb[1]);
  NLINV_ADV(float2, part);
  NLINV_ADV(float2, Hr);
  NLINV_ADV(float2, vold);
  NLINV_ADV(float2, sb[0]);
  NLINV_ADV(float2, sb[1]);
  NLINV_ADV(float2, Hw);
  NLINV_ADV(float2, Hs);
  NLINV_ADV(double, cgs);
#undef NLINV_ADV
  return C;
}

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

inline int plan_grid(int items, int min_items) {
  int g = items > min_items ? items : min_items;
  if (g < 1) g = 1;
  return g > kMaxPart ? kMaxPart : g;
}

}  // namespace nlinv

// ================================================================== plan
// ================================================================== plan
struct nlinv_plan_s {
  nlinv_params_t prm;
  int N, G, Gc, J, U;
  long long nx;
  int dev, nsm;
  int max_batch = 1;
  size_t fstride = 0;         // bytes between the per-frame workspaces
  void* mem = nullptr;
  void* prep = nullptr;
  size_t prep_bytes = 0;
  nlinv::Ctx C;               // frame 0's workspace
  float* psf;
  int coop_grid = 0;          // co-resident CTAs of k_frame
  int batch_occ = 0;          // co-resident CTAs per SM of k_batch
  int cl_cs = 0;              // CTAs per cluster of k_frame_cl (0: it does not fit)
  nlinv::cl::Lay cl_lay;             // its shared-memory layout
  // per-phase execution (exec_mode 0, 1, 4): CTAs per frame of a one-phase
  // launch, the device table of the frames' inputs and outputs that the
  // phase kernels read, and the phase sequences captured into CUDA graphs
  // (one per frame count and alpha_0)
  int phase_grid = 0;
  int colc_grid = 0;          // CTAs per frame of the CG's PSF column pass (no partial sums)
  bool dense = false;         // a lone frame has work for two CTAs per SM (runs like a batch)
  int op_minb = 1;            // CTAs per SM of the operator kernels (Cfg::OMINB)
  int op_grid = 0;            // cap on the CTAs of an operator launch (0: one per item)
  nlinv::FrameIO* io_dev = nullptr;
  cudaStream_t gcap = nullptr;
  struct PhaseGraph {
    int nf = 0;
    double alpha0 = 0.0;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<PhaseGraph> pgraphs;
  // reverse passes: one stream, completion event, captured graph and staging
  // buffers per frame slot of a batch, and their own workspace allocation
  std::vector<cudaStream_t> vjp_st;
  std::vector<cudaEvent_t> vjp_ev;
  cudaEvent_t vjp_fork = nullptr;
  double* vjp_host = nullptr;  // pinned: alpha0-bar and breakdown flags
  void* vjp_mem = nullptr;     // slots' workspaces, then the gather area
  size_t vjp_bytes = 0;
  struct VjpGraph {
    cudaGraphExec_t exec = nullptr;
    double alpha0 = 0.0;
    int turn = -1, has_xprev = -1, want_xprev_bar = -1;
    void* stage = nullptr;     // Y, Y-bar [J][G][G]; gbar, x_prev, x_prev-bar [n_x]
  };
  std::vector<VjpGraph> vjp_graphs;
  cudaStream_t aux = nullptr; // stream of this plan's group inside nlinv_batch
  cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
};

namespace nlinv {

// Operations of one FFT grid size, implemented by grid.cu for its Cfg.
// Every call is asynchronous on `st` and returns NLINV_OK or an error code.
struct GridOps {
  int G, N;
  // per plan: kernel attributes, co-residency of the persistent kernels and
  // (exec_mode 0 or 3) the cluster kernel's configuration
  int (*setup)(nlinv_plan_s* pl);
  // for callers without a plan set-up: kernel attributes and the constant
  // tables of this unit on the current device
  int (*prepare)();
  // coil maps c = W^-1 c^ of x into the plan's coil buffer
  int (*coils)(const nlinv_plan_s* pl, cudaStream_t st, const float2* x);
  // z = DF(x)[d], dx = DF(x)^H z, out = (DF^H P DF + alpha) d at x; with
  // coils_ready the plan's coil buffer already holds W^-1 of x's coil part
  int (*DF)(const nlinv_plan_s* pl, cudaStream_t st, const float2* x, const float2* d, float2* z,
            bool coils_ready);
  int (*DFH)(const nlinv_plan_s* pl, cudaStream_t st, const float2* x, const float2* z, float2* out,
             bool coils_ready);
  int (*normal)(const nlinv_plan_s* pl, cudaStream_t st, const float2* x, const float2* d, const float* P,
                double alpha, float2* out, bool coils_ready);
  // Y = U pad(img), img [J][N][N] in the plan's s buffer (gridding's last step)
  int (*grid_fwd)(const nlinv_plan_s* pl, cudaStream_t st, float2* Y);
  // convolution gridding after the spreading: Y = U pad(scale dap dap crop U^H Z),
  // Z [J][G][G] the spread grid, dap [N] the per-axis deapodisation
  int (*grid_kb)(const nlinv_plan_s* pl, cudaStream_t st, const float2* Z, const float* dap, float scale,
                 float2* Y);
  // one whole frame on the plan's execution path
  int (*frame)(const nlinv_plan_s* pl, cudaStream_t st, const FrameArgs& F);
  // frames of one plan together: one launch per phase over all frames
  // (exec_mode 0, 1, 4, when no frame waits for another), else one
  // cooperative launch of `grid` CTAs
  int (*batch)(const nlinv_plan_s* pl, cudaStream_t st, const BatchArgs& B, int grid);
#ifdef NLINV_TIMELINE
  int (*timeline)(unsigned long long* host, int n);
  int (*stages)(unsigned long long* ns, unsigned long long* cnt);
#endif
};

// The compiled grids X(G1, G2, N, TW, MINB): G = G1 x G2 with an N x N field
// of view, tile width TW and MINB CTAs per SM (Cfg in phases.cuh); one
// grid.cu unit each.  G = 2N for the twofold grids; the others are grids
// G = 2 gamma N of Eq. (8) with gamma > 1 (radix 3, 5 and 7 splits).  A unit
// left out of a build leaves its grid unsupported (weak reference).  The
// tile widths are measured picks (tune.py and the bench): 12 at 320 for one
// frame at a time; 8 at 384 (192-thread CTAs, two per SM) for frames in
// flight together (the 384^2 / 16-channel class of the batched workload:
// 493 -> 522 frames/s over the three classes); 8 at 512, where a 64-channel
// frame is dense enough to run like a batch (26.0 against 27.2 ms per frame
// with 16-wide tiles at one CTA per SM).
#define NLINV_GRIDS(X)                                                                               \
  X(4, 4, 8, 16, 2) X(4, 6, 12, 16, 2) X(4, 10, 20, 16, 2) X(8, 8, 32, 16, 2) X(8, 16, 64, 16, 2)   \
  X(16, 16, 128, 16, 2) X(16, 20, 160, 12, 1) X(16, 24, 192, 8, 1) X(16, 32, 256, 8, 1)           \
  X(4, 14, 20, 16, 2) X(6, 9, 20, 16, 2) X(8, 9, 24, 16, 2) X(16, 28, 160, 16, 1)                  \
  X(16, 30, 160, 16, 1) X(18, 27, 160, 16, 1) X(16, 32, 160, 16, 1) X(20, 28, 160, 16, 1)          \
  X(16, 24, 128, 16, 1)
#define NLINV_DECLARE_OPS(a, b, n, tw, mb) const GridOps* grid_ops_##a##_##b##_##n() __attribute__((weak));
NLINV_GRIDS(NLINV_DECLARE_OPS)
#undef NLINV_DECLARE_OPS

// the operations of grid G with an N x N field of view, or nullptr when that
// pair has no compiled schedule
const GridOps* grid_ops(int G, int N);

}  // namespace nlinv
