// C-ABI implementation of the GB300 NLINV hot path (see include/nlinv.h).
//
// Kernels: the fused phases of phases.cuh, launched either one per phase or
// all inside one persistent cooperative kernel per frame (grid barriers with
// bounded waits between phases), plus the preprocessing kernels that turn a
// trajectory into a PSF and raw samples into gridded data.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "nlinv.h"
#include "phases.cuh"

using namespace nlinv;

namespace {

// ------------------------------------------------------------ errors
thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? NLINV_ENOMEM : NLINV_ECUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

#define CKL(what)                                  \
  do {                                             \
    cudaError_t e_ = cudaGetLastError();           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// ---------------------------------------------------- kernel wrappers
// every CTA of a one-frame launch works on that frame
__device__ __forceinline__ Ctx whole_grid(const Ctx& C0) {
  Ctx C = C0;
  C.bid = blockIdx.x;
  C.nb = gridDim.x;
  return C;
}

template <class K>
__global__ void __launch_bounds__(K::BS) k_coil_y(Ctx C0, const float2* src, float2* hout) {
  const Ctx C = whole_grid(C0);
  extern __shared__ float2 sm[];
  phase_coil_y<K>(C, sm, src, hout);
}

template <class K>
__global__ void __launch_bounds__(K::BS) k_row_cg(Ctx C0, int k, const float2* p_old, float2* p_new,
                                                  float2* vout) {
  const Ctx C = whole_grid(C0);
  extern __shared__ float2 sm[];
  __shared__ float2 sred[32];
  phase_row_cg<K>(C, sm, sred, k, p_old, p_new, vout);
}

template <class K>
__global__ void __launch_bounds__(K::BS) k_row_b(Ctx C0, int mode, const float2* hin, const float2* rho,
                                                 const float2* drho, const float2* img, float2* vout) {
  const Ctx C = whole_grid(C0);
  extern __shared__ float2 sm[];
  phase_row_b<K>(C, sm, mode, hin, rho, drho, img, vout);
}

template <class K>
__global__ void __launch_bounds__(K::BS) k_col_c(Ctx C0, int mode, const float* P, const float2* Yin,
                                                 float2* zout, float2* vio, int k) {
  const Ctx C = whole_grid(C0);
  extern __shared__ float2 sm[];
  phase_col_c<K>(C, sm, mode, P, Yin, zout, vio, k);
}

template <class K>
__global__ void __launch_bounds__(K::BS) k_row_d(Ctx C0, const float2* rho, const float2* win, float2* sout,
                                                 float2* kbout) {
  const Ctx C = whole_grid(C0);
  extern __shared__ float2 sm[];
  phase_row_d<K>(C, sm, rho, win, sout, kbout);
}

template <class K>
__global__ void __launch_bounds__(K::BS) k_col_e(Ctx C0, int mode, float alpha, int k, const float2* kbin,
                                                 const float2* sin, const float2* p_old, float2* p_new,
                                                 float2* out, float2* hout, int slot) {
  const Ctx C = whole_grid(C0);
  extern __shared__ float2 sm[];
  __shared__ float2 sred[32];
  switch (mode) {
    case E_CG: phase_col_e<K, E_CG>(C, sm, sred, alpha, k, kbin, sin, p_old, p_new, out, hout, slot); break;
    case E_RHS: phase_col_e<K, E_RHS>(C, sm, sred, alpha, k, kbin, sin, p_old, p_new, out, hout, slot); break;
    case E_DFH: phase_col_e<K, E_DFH>(C, sm, sred, alpha, k, kbin, sin, p_old, p_new, out, hout, slot); break;
    default: phase_col_e<K, E_NORMAL>(C, sm, sred, alpha, k, kbin, sin, p_old, p_new, out, hout, slot);
  }
}

template <class K>
__global__ void __launch_bounds__(K::BS) k_upd(Ctx C0, int k, int last, const float2* p) {
  const Ctx C = whole_grid(C0);
  extern __shared__ float2 sm[];
  __shared__ float2 sred[32];
  phase_upd<K>(C, sm, sred, k, last != 0, p);
}

__global__ void k_init(Ctx C0, const float2* xprev, float damping) {
  const Ctx C = whole_grid(C0);
  phase_init(C, xprev, damping);
}

__global__ void k_final(Ctx C0, float2* xout, float2* rho_out, float2* img_out) {
  const Ctx C = whole_grid(C0);
  phase_final(C, xout, rho_out, img_out);
}

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
#undef NLINV_ADV
  return C;
}

#ifdef NLINV_TIMELINE
// profiling builds: per-CTA global timer at the start of every phase and
// after every barrier of the first frame launch
__device__ unsigned long long g_timeline[160][1024];
__device__ __forceinline__ void tl_mark(int& i) {
  if (threadIdx.x == 0 && blockIdx.x < 160 && i < 1024) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    g_timeline[blockIdx.x][i] = t;
  }
  ++i;
}
#define NLINV_MARK() tl_mark(tl_i)
#else
#define NLINV_MARK()
#endif

// Every phase of every Newton step and CG iteration of one frame, separated
// by bounded grid barriers (which all CTAs of the launch pass together).

// The five phases of a Newton step's right-hand side (Eqs. (2)-(3): DF^H (Y -
// P F^(x^_n)) - alpha_n (x^_n - x_ref), and H r_0).  They run once per Newton
// step against ten CG iterations, so they live in their own function: kept
// out of the persistent kernel's body, they no longer add to the register
// pressure (and spills) of the CG loop, which measured 2 % faster per frame.
template <class K>
__device__ __noinline__ bool newton_rhs_phases(const Ctx& C, float2* sm, float2* sred, const FrameIO& io, float al,
                                               bool lastreg, float damping, unsigned& epoch) {
  const int NN = C.N * C.N;
  phase_coil_y<K>(C, sm, C.xn + NN, C.h);
  if (!grid_sync(C, epoch)) return false;
  phase_row_b<K>(C, sm, ROW_COIL, C.h, C.xn, nullptr, nullptr, C.v);
  if (!grid_sync(C, epoch)) return false;
  phase_col_c<K>(C, sm, COL_RHS, io.P, io.Y, nullptr, C.v);
  if (!grid_sync(C, epoch)) return false;
  phase_row_d<K>(C, sm, C.xn, C.v, C.s, C.kb);
  if (!grid_sync(C, epoch)) return false;
  phase_col_e<K, E_RHS>(C, sm, sred, al, 0, C.kb, C.s, nullptr, nullptr, C.rb[0], C.Hr, SLOT_RR0,
                        lastreg ? io.xlast : nullptr, lastreg ? damping : 1.f);
  if (!grid_sync(C, epoch)) return false;
  return true;
}

template <class K>
__device__ __forceinline__ void frame_body(const Ctx& C, float2* sm, float2* sred, const FrameIO& io, int M,
                                           int Kcg, float damping, const float* alpha) {
  const int NN = C.N * C.N;
  unsigned epoch = 0;
#ifdef NLINV_TIMELINE
  int tl_i = 0;
#endif
#define NLINV_SYNC()              \
  NLINV_MARK();                   \
  if (!grid_sync(C, epoch)) return; \
  NLINV_MARK()
  phase_init(C, io.xprev, damping);
  NLINV_SYNC();
  for (int n = 0; n < M; ++n) {
    const float al = alpha[n];
    const bool lastreg = (n == M - 1) && io.xlast != nullptr;
    if (lastreg && io.wait) {   // Eq. (10): the last step waits for frame n - 1
      if (threadIdx.x == 0) {
        long long it = 0;
        while (ld_acquire(io.wait) == 0u) {
          if (*(volatile int*)C.err != 0) break;
          if (++it > C.spin_limit) {
            raise_err(C, DEV_ETIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      if (*(volatile int*)C.err != 0) return;
    }
    // Newton right-hand side: DF^H (Y - P F^(x^_n)) - alpha_n (x^_n - x_ref)
    if (!newton_rhs_phases<K>(C, sm, sred, io, al, lastreg, damping, epoch)) return;
    for (int k = 0; k < Kcg; ++k) {
      float2* pk = C.pb[k & 1];
      const float2* pm = C.pb[(k + 1) & 1];
      phase_row_cg<K>(C, sm, sred, k, pm, pk, C.v);
      NLINV_SYNC();
      phase_col_cg<K>(C, sm, io.P, C.v, k);
      NLINV_SYNC();
      phase_row_d<K>(C, sm, C.xn, C.v, C.s, C.kb);
      NLINV_SYNC();
      phase_col_e<K, E_CG>(C, sm, sred, al, k, C.kb, C.s, pm, pk, C.q, nullptr, SLOT_PQ);
      NLINV_SYNC();
      phase_upd<K>(C, sm, sred, k, k == Kcg - 1, pk);
      NLINV_SYNC();
    }
  }
  phase_coil_y<K>(C, sm, C.xn + NN, C.h);
  NLINV_SYNC();
  phase_row_b<K>(C, sm, ROW_COILONLY, C.h, nullptr, nullptr, nullptr, nullptr);
  NLINV_SYNC();
  phase_final(C, io.xout, io.rho_out, io.img_out);
  if (io.done) {   // publish x_out to a frame waiting on this one
    NLINV_SYNC();
    if (C.bid == 0 && threadIdx.x == 0) st_release(io.done, 1u);
  }
#undef NLINV_SYNC
}

// One whole NLINV frame in one cooperative launch.
template <class K>
__global__ void __launch_bounds__(K::BS, K::MINB) k_frame(Ctx C0, FrameArgs F) {
  extern __shared__ float2 sm[];
  __shared__ float2 sred[32];
  const Ctx C = whole_grid(C0);
  frame_body<K>(C, sm, sred, F.io, F.M, F.K, F.damping, F.alpha);
}

// Several frames of one size in one cooperative launch: the CTAs are split
// into one contiguous group per frame; each group runs its frame on its own
// workspace with its own barrier, so the groups progress independently (a
// frame whose last Newton step waits for an earlier frame of the launch
// cannot hold the others up: all groups are co-resident).
template <class K>
__global__ void __launch_bounds__(K::BS, K::MINB) k_batch(Ctx C0, BatchArgs B) {
  extern __shared__ float2 sm[];
  __shared__ float2 sred[32];
  const int nf = B.nf;
  const int f = (int)(((long long)blockIdx.x * nf) / gridDim.x);
  const int lo = (int)(((long long)f * gridDim.x + nf - 1) / nf);
  const int hi = (int)(((long long)(f + 1) * gridDim.x + nf - 1) / nf);
  Ctx C = frame_ctx(C0, (size_t)f * B.fstride);
  C.bid = blockIdx.x - lo;
  C.nb = hi - lo;
  C.bar = C0.bar + (size_t)f * kBarStride;   // this group's own barrier
  frame_body<K>(C, sm, sred, B.io[f], B.M, B.K, B.damping, B.alpha);
}

// bounded wait on a device flag (used to test the timeout path)
__global__ void k_wait_flag(const volatile int* flag, int expected, long long limit, int* err) {
  if (threadIdx.x != 0) return;
  long long it = 0;
  while (*flag != expected) {
    if (++it > limit) {
      atomicCAS(err, 0, NLINV_ETIMEOUT);
      return;
    }
    __nanosleep(100);
  }
}

// ----------------------------------------------- preprocessing kernels
// Dirichlet kernel tables Dx[s][f] = Dir(kx_s - f/G), Dy likewise (FP64 math)
__global__ void k_dirichlet(int N, int G, int S, const double* __restrict__ kxy, float* Dx, float* Dy) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * G) return;
  const int s = idx / G, f = idx - s * G;
  const double ff = (double)f / G, m = 2.0 * N - 1.0;
#pragma unroll
  for (int ax = 0; ax < 2; ++ax) {
    const double tt = kxy[2 * s + ax] - ff;
    const double r = tt - rint(tt);
    const double val = (r == 0.0) ? m : sinpi(m * r) / sinpi(r);
    (ax ? Dy : Dx)[idx] = (float)val;
  }
}

// P[fy][fx] = scale * sum_s Dy[s][fy] Dx[s][fx]   (FP64 accumulation)
__global__ void k_psf_gemm(int G, int S, const float* __restrict__ Dx, const float* __restrict__ Dy, float* P,
                           double scale) {
  __shared__ float ay[16][17], ax[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int fx = blockIdx.x * 16 + tx, fy = blockIdx.y * 16 + ty;
  const int fyl = blockIdx.y * 16 + tx;
  double acc = 0.0;
  for (int s0 = 0; s0 < S; s0 += 16) {
    const int s = s0 + ty;
    ay[ty][tx] = (s < S && fyl < G) ? Dy[(size_t)s * G + fyl] : 0.f;
    ax[ty][tx] = (s < S && fx < G) ? Dx[(size_t)s * G + fx] : 0.f;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) acc = fma((double)ay[u][ty], (double)ax[u][tx], acc);
    __syncthreads();
  }
  if (fx < G && fy < G) P[(size_t)fy * G + fx] = (float)(acc * scale);
}

// E[s][r] = exp(+2 pi i k_s r), phase reduced mod 1 in FP64
__global__ void k_ndft_tables(int N, int S, const double* __restrict__ kxy, float2* Ex, float2* Ey) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * N) return;
  const int s = idx / N, r = idx - s * N;
#pragma unroll
  for (int ax = 0; ax < 2; ++ax) {
    const double tt = kxy[2 * s + ax] * r;
    const double fr = tt - rint(tt);
    double sn, cs;
    sincospi(2.0 * fr, &sn, &cs);
    (ax ? Ey : Ex)[idx] = make_float2((float)cs, (float)sn);
  }
}

// img[j][y][x] = scale * sum_s y[j][s] Ey[s][y] Ex[s][x]
__global__ void k_adj_ndft(int N, int S, const float2* __restrict__ yv, const float2* __restrict__ Ex,
                           const float2* __restrict__ Ey, float2* img, float scale) {
  __shared__ float2 A[16][17], B[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y, j = blockIdx.z;
  const int x = blockIdx.x * 16 + tx, y = blockIdx.y * 16 + ty;
  const int yl = blockIdx.y * 16 + tx;
  float2 acc = czero();
  for (int s0 = 0; s0 < S; s0 += 16) {
    const int s = s0 + ty;
    float2 a = czero(), b = czero();
    if (s < S) {
      if (yl < N) a = cmul(yv[(size_t)j * S + s], Ey[(size_t)s * N + yl]);
      if (x < N) b = Ex[(size_t)s * N + x];
    }
    A[ty][tx] = a;
    B[ty][tx] = b;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const float2 p = A[u][ty], q = B[u][tx];
      acc.x = fmaf(p.x, q.x, fmaf(-p.y, q.y, acc.x));
      acc.y = fmaf(p.x, q.y, fmaf(p.y, q.x, acc.y));
    }
    __syncthreads();
  }
  if (x < N && y < N) img[((size_t)j * N + y) * N + x] = cscale(acc, scale);
}

// ----------------------------------------------------- size dispatch
// NLINV_ONLY_G=<G> compiles one grid size only (quick profiling builds)
#ifdef NLINV_ONLY_G
#define NLINV_CASE(g, a, b)                          \
  case g:                                            \
    if constexpr (g == NLINV_ONLY_G) return f(Cfg<a, b>{}); \
    else return NLINV_EUNSUPPORTED;
#else
#define NLINV_CASE(g, a, b) \
  case g: return f(Cfg<a, b>{});
#endif
template <class F>
int dispatch(int G, F&& f) {
  switch (G) {
    NLINV_CASE(16, 4, 4)
    NLINV_CASE(24, 4, 6)
    NLINV_CASE(40, 4, 10)
    NLINV_CASE(64, 8, 8)
    NLINV_CASE(128, 8, 16)
    NLINV_CASE(256, 16, 16)
    NLINV_CASE(320, 16, 20)
    NLINV_CASE(384, 16, 24)
    NLINV_CASE(512, 16, 32)
    default: return NLINV_EUNSUPPORTED;
  }
}

bool supported_grid(int G) {
  return dispatch(G, [](auto) { return NLINV_OK; }) == NLINV_OK;
}

std::mutex g_mu;
bool g_tw_ready[64] = {};

int ensure_constants(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return NLINV_EINVAL;
  if (g_tw_ready[dev]) return NLINV_OK;
  float2 h[TWL];
  for (int e = 0; e < TWL; ++e) {
    const double a = -2.0 * M_PI * (double)e / TWL;
    h[e] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  CK(cudaMemcpyToSymbol(c_tw, h, sizeof(h)));
  g_tw_ready[dev] = true;
  return NLINV_OK;
}

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

}  // namespace

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
  Ctx C;                      // frame 0's workspace
  float* psf;
  int coop_grid = 0;          // co-resident CTAs of k_frame
  int batch_occ = 0;          // co-resident CTAs per SM of k_batch
  cudaStream_t aux = nullptr; // stream of this plan's group inside nlinv_batch
  cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
};

namespace {

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

int plan_grid(int items, int min_items) {
  int g = items > min_items ? items : min_items;
  if (g < 1) g = 1;
  return g > kMaxPart ? kMaxPart : g;
}

template <class K>
int set_smem_attrs() {
  if (K::SMEM > 48 * 1024) {
    CK(cudaFuncSetAttribute(k_coil_y<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_row_b<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_col_c<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_row_d<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_col_e<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_row_cg<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_upd<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_frame<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_batch<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
  }
  return NLINV_OK;
}

// launch helpers for the one-launch-per-phase path
template <class K>
struct Launch {
  const nlinv_plan_s* pl;
  cudaStream_t st;
  int fixed = 0;   // if > 0: every launch uses this many CTAs (CG reductions need equal counts)
  int pick(int g) const { return fixed > 0 ? fixed : g; }
  int coil_y(const float2* src, float2* hout) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.Gc + K::TW - 1) / K::TW), 1);
    k_coil_y<K><<<pick(g), K::BS, K::SMEM, st>>>(C, src, hout);
    CKL("k_coil_y");
    return NLINV_OK;
  }
  int row_cg(int k, const float2* p_old, float2* p_new, float2* vout) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.N + K::TW - 1) / K::TW), 1);
    k_row_cg<K><<<pick(g), K::BS, K::SMEM, st>>>(C, k, p_old, p_new, vout);
    CKL("k_row_cg");
    return NLINV_OK;
  }
  int row_b(int mode, const float2* hin, const float2* rho, const float2* drho, const float2* img,
            float2* vout) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.N + K::TW - 1) / K::TW), 1);
    k_row_b<K><<<pick(g), K::BS, K::SMEM, st>>>(C, mode, hin, rho, drho, img, vout);
    CKL("k_row_b");
    return NLINV_OK;
  }
  int col_c(int mode, const float* P, const float2* Yin, float2* zout, float2* vio, int k = 0) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.G + K::TW - 1) / K::TW), 1);
    k_col_c<K><<<pick(g), K::BS, K::SMEM, st>>>(C, mode, P, Yin, zout, vio, k);
    CKL("k_col_c");
    return NLINV_OK;
  }
  int row_d(const float2* rho, const float2* win, float2* sout, float2* kbout) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.N + K::TW - 1) / K::TW), 1);
    k_row_d<K><<<pick(g), K::BS, K::SMEM, st>>>(C, rho, win, sout, kbout);
    CKL("k_row_d");
    return NLINV_OK;
  }
  int col_e(int mode, float alpha, int k, const float2* kbin, const float2* sin, const float2* p_old,
            float2* p_new, float2* out, float2* hout, int slot) const {
    const Ctx& C = pl->C;
    const int items = C.J * ((C.Gc + K::TW - 1) / K::TW);
    const int g = plan_grid(items, (C.N * C.N + K::BS - 1) / K::BS);
    k_col_e<K><<<pick(g), K::BS, K::SMEM, st>>>(C, mode, alpha, k, kbin, sin, p_old, p_new, out, hout, slot);
    CKL("k_col_e");
    return NLINV_OK;
  }
  int upd(int k, int last, const float2* p) const {
    const Ctx& C = pl->C;
    const int items = C.J * ((C.Gc + K::TW - 1) / K::TW);
    const int g = plan_grid(items, (C.N * C.N + K::BS - 1) / K::BS);
    k_upd<K><<<pick(g), K::BS, K::SMEM, st>>>(C, k, last, p);
    CKL("k_upd");
    return NLINV_OK;
  }
  // coil maps c_j = W^-1 c^_j of x^ into the plan's c buffer
  int coils(const float2* xhat) const {
    const Ctx& C = pl->C;
    int rc = coil_y(xhat + (size_t)C.N * C.N, C.h);
    if (rc) return rc;
    return row_b(ROW_COILONLY, C.h, nullptr, nullptr, nullptr, nullptr);
  }
};

#define RC(x)                 \
  do {                        \
    int rc_ = (x);            \
    if (rc_ != NLINV_OK) return rc_; \
  } while (0)

int check_plan(const nlinv_plan_s* pl) { return pl ? NLINV_OK : NLINV_EINVAL; }

}  // namespace

extern "C" {

const char* nlinv_strerror(int code) {
  switch (code) {
    case NLINV_OK: return "ok";
    case NLINV_EINVAL: return "invalid argument";
    case NLINV_ECUDA: return "CUDA runtime error";
    case NLINV_ENOMEM: return "out of device memory";
    case NLINV_ETIMEOUT: return "bounded device wait expired";
    case NLINV_ENUMERIC: return "CG breakdown (Re<p,Ap> <= 0 or not finite)";
    case NLINV_EUNSUPPORTED: return "unsupported grid size";
    default: return "unknown error";
  }
}

const char* nlinv_last_cuda_error(void) { return g_cuda_err; }

int nlinv_default_params(nlinv_params_t* p, int N, int J) {
  if (!p || N <= 0 || J <= 0) return NLINV_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->N = N;
  p->J = J;
  p->Gc = 0;
  p->newton_steps = 7;
  p->cg_iters = 10;
  p->n_turns = 1;
  p->alpha0 = 1.0;
  p->q = 0.5;
  p->damping = 1.0;
  p->w_a = 220.0;
  p->w_l = 32.0;
  p->spin_limit = 0;
  p->exec_mode = 0;
  p->max_batch = 1;
  return NLINV_OK;
}

int nlinv_plan(nlinv_plan_t* out, const nlinv_params_t* p, const float* psf, nlinv_stream_t stream) {
  if (!out || !p) return NLINV_EINVAL;
  *out = nullptr;
  const int N = p->N, G = 2 * p->N, J = p->J;
  const int Gc = p->Gc ? p->Gc : G / 4;
  if (N <= 0 || J <= 0 || J > 4096) return NLINV_EINVAL;
  if (!supported_grid(G)) return NLINV_EUNSUPPORTED;
  if (Gc < 2 || Gc > G || (Gc & 1)) return NLINV_EINVAL;
  if (p->newton_steps < 1 || p->newton_steps > kMaxNewton) return NLINV_EINVAL;
  if (p->cg_iters < 0 || p->cg_iters > 4096) return NLINV_EINVAL;
  if (p->n_turns < 1 || p->n_turns > 1024) return NLINV_EINVAL;
  if (!(p->alpha0 > 0.0) || !(p->q > 0.0) || p->q > 1.0 || !(p->damping >= 0.0)) return NLINV_EINVAL;
  if (!(p->w_a >= 0.0) || !(p->w_l >= 0.0)) return NLINV_EINVAL;
  if (p->exec_mode != 0 && p->exec_mode != 1) return NLINV_EINVAL;
  if (p->max_batch < 0 || p->max_batch > kMaxBatch) return NLINV_EINVAL;
  if (psf && ((uintptr_t)psf & 3u)) return NLINV_EINVAL;

  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  RC(ensure_constants(dev));

  nlinv_plan_s* pl = new nlinv_plan_s();
  pl->prm = *p;
  pl->prm.Gc = Gc;
  if (pl->prm.spin_limit <= 0) pl->prm.spin_limit = 1LL << 22;
  pl->N = N;
  pl->G = G;
  pl->Gc = Gc;
  pl->J = J;
  pl->U = p->n_turns;
  pl->max_batch = p->max_batch > 0 ? p->max_batch : 1;
  pl->nx = (long long)N * N + (long long)J * Gc * Gc;
  pl->dev = dev;
  cudaError_t e = cudaDeviceGetAttribute(&pl->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }

  // one allocation: shared tables, then max_batch per-frame workspaces
  const size_t f2 = sizeof(float2);
  const size_t nx = (size_t)pl->nx;
  size_t off[40];
  size_t tot = 0;
  int nb = 0;
  auto take = [&](size_t bytes) {
    off[nb++] = tot;
    tot += align_up(bytes);
  };
  take(G * f2);                          // 0 tw
  take((size_t)Gc * Gc * sizeof(float)); // 1 dinv
  take((size_t)pl->U * G * G * sizeof(float));  // 2 psf
  take(sizeof(int));                     // 3 err
  take((size_t)kMaxBatch * kBarStride * sizeof(unsigned));  // 4 barrier counters and flags
  const size_t shared_bytes = tot;
  take((size_t)J * N * N * f2);          // 5 c
  take((size_t)J * N * Gc * f2);         // 6 h
  take((size_t)J * N * G * f2);          // 7 v
  take((size_t)J * N * N * f2);          // 8 s
  take((size_t)J * N * Gc * f2);         // 9 kb
  for (int i = 0; i < 7; ++i) take(nx * f2);  // 10..16 xn xref xcg r q p0 p1
  take((size_t)NSLOT * kMaxPart * sizeof(float2));  // 17 part
  take(nx * f2);                         // 18 r1 (second residual buffer)
  take((size_t)J * N * Gc * f2);         // 19 Hr
  take((size_t)J * N * G * f2);          // 20 vold
  pl->fstride = tot - shared_bytes;
  tot = shared_bytes + pl->fstride * (size_t)pl->max_batch;
  e = cudaMalloc(&pl->mem, tot);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaMalloc(plan)");
  }
  char* base = (char*)pl->mem;
  Ctx& C = pl->C;
  std::memset(&C, 0, sizeof(C));
  C.N = N;
  C.G = G;
  C.Gc = Gc;
  C.J = J;
  C.nx = (int)nx;
  C.U = pl->U;
  C.inv_G = (float)(1.0 / G);
  C.inv_G2 = (float)(1.0 / ((double)G * G));
  C.tw = (const float2*)(base + off[0]);
  C.dinv = (const float*)(base + off[1]);
  pl->psf = (float*)(base + off[2]);
  C.psf = pl->psf;
  C.err = (int*)(base + off[3]);
  C.bar = (unsigned*)(base + off[4]);
  C.c = (float2*)(base + off[5]);
  C.h = (float2*)(base + off[6]);
  C.v = (float2*)(base + off[7]);
  C.s = (float2*)(base + off[8]);
  C.kb = (float2*)(base + off[9]);
  C.xn = (float2*)(base + off[10]);
  C.xref = (float2*)(base + off[11]);
  C.xcg = (float2*)(base + off[12]);
  C.rb[0] = (float2*)(base + off[13]);
  C.rb[1] = (float2*)(base + off[18]);
  C.q = (float2*)(base + off[14]);
  C.pb[0] = (float2*)(base + off[15]);
  C.pb[1] = (float2*)(base + off[16]);
  C.part = (float2*)(base + off[17]);
  C.Hr = (float2*)(base + off[19]);
  C.vold = (float2*)(base + off[20]);
  C.spin_limit = pl->prm.spin_limit;

  // host tables in FP64, rounded once
  std::vector<float2> tw(G);
  for (int k = 0; k < G; ++k) {
    const double a = -2.0 * M_PI * (double)k / G;
    tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  std::vector<float> dinv((size_t)Gc * Gc);
  for (int iy = 0; iy < Gc; ++iy) {
    const int fy = iy < (Gc + 1) / 2 ? iy : iy - Gc;
    for (int ix = 0; ix < Gc; ++ix) {
      const int fx = ix < (Gc + 1) / 2 ? ix : ix - Gc;
      const double ky = 2.0 * fy / G, kx = 2.0 * fx / G;
      dinv[(size_t)iy * Gc + ix] = (float)std::pow(1.0 + p->w_a * (kx * kx + ky * ky), -p->w_l / 2.0);
    }
  }
  int rc = NLINV_OK;
  auto fail = [&](int code) {
    cudaFree(pl->mem);
    delete pl;
    return code;
  };
  if ((e = cudaMemsetAsync(pl->mem, 0, tot, st)) != cudaSuccess) return fail(cuda_fail(e, "memset"));
  if ((e = cudaMemcpyAsync((void*)C.tw, tw.data(), G * f2, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail(cuda_fail(e, "tw"));
  if ((e = cudaMemcpyAsync((void*)C.dinv, dinv.data(), dinv.size() * sizeof(float), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return fail(cuda_fail(e, "dinv"));
  if (psf) {
    if ((e = cudaMemcpyAsync(pl->psf, psf, (size_t)pl->U * G * G * sizeof(float), cudaMemcpyDeviceToDevice,
                             st)) != cudaSuccess)
      return fail(cuda_fail(e, "psf"));
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(cuda_fail(e, "sync"));

  rc = dispatch(G, [&](auto k) -> int {
    using K = decltype(k);
    RC(set_smem_attrs<K>());
    int nbk = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, k_frame<K>, K::BS, K::SMEM));
    int g = nbk * pl->nsm;
    if (g > kMaxPart) g = kMaxPart;
    pl->coop_grid = g;
    int nbb = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbb, k_batch<K>, K::BS, K::SMEM));
    pl->batch_occ = nbb;
    CK(cudaStreamCreateWithFlags(&pl->aux, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&pl->ev_done, cudaEventDisableTiming));
    return (g > 0 && nbb > 0) ? NLINV_OK : NLINV_ECUDA;
  });
  if (rc != NLINV_OK) return fail(rc);
  *out = pl;
  return NLINV_OK;
}

int nlinv_plan_destroy(nlinv_plan_t pl) {
  if (!pl) return NLINV_EINVAL;
  if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
  if (pl->ev_done) cudaEventDestroy(pl->ev_done);
  if (pl->aux) cudaStreamDestroy(pl->aux);
  cudaFree(pl->prep);
  cudaError_t e = cudaFree(pl->mem);
  delete pl;
  return e == cudaSuccess ? NLINV_OK : cuda_fail(e, "cudaFree");
}

int nlinv_plan_sizes(nlinv_plan_t pl, long long* nx, int* G, int* Gc) {
  RC(check_plan(pl));
  if (nx) *nx = pl->nx;
  if (G) *G = pl->G;
  if (Gc) *Gc = pl->Gc;
  return NLINV_OK;
}

int nlinv_set_psf(nlinv_plan_t pl, int turn, const float* psf, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!psf || turn < 0 || turn >= pl->U || ((uintptr_t)psf & 3u)) return NLINV_EINVAL;
  const size_t bytes = (size_t)pl->G * pl->G * sizeof(float);
  CK(cudaMemcpyAsync(pl->psf + (size_t)turn * pl->G * pl->G, psf, bytes, cudaMemcpyDeviceToDevice,
                     (cudaStream_t)stream));
  return NLINV_OK;
}

static int ensure_prep(nlinv_plan_s* pl, size_t bytes) {
  if (pl->prep_bytes >= bytes) return NLINV_OK;
  if (pl->prep) {
    CK(cudaFree(pl->prep));
    pl->prep = nullptr;
    pl->prep_bytes = 0;
  }
  CK(cudaMalloc(&pl->prep, bytes));
  pl->prep_bytes = bytes;
  return NLINV_OK;
}

int nlinv_psf(nlinv_plan_t pl, int turn, int S, const double* kxy, float* P_out, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (turn < 0 || turn >= pl->U || S <= 0 || !kxy || ((uintptr_t)kxy & 7u)) return NLINV_EINVAL;
  if (P_out && ((uintptr_t)P_out & 3u)) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int G = pl->G;
  RC(ensure_prep(pl, (size_t)2 * S * G * sizeof(float)));
  float* Dx = (float*)pl->prep;
  float* Dy = Dx + (size_t)S * G;
  const int tot = S * G;
  k_dirichlet<<<(tot + 255) / 256, 256, 0, st>>>(pl->N, G, S, kxy, Dx, Dy);
  CKL("k_dirichlet");
  float* P = pl->psf + (size_t)turn * G * G;
  k_psf_gemm<<<dim3((G + 15) / 16, (G + 15) / 16), dim3(16, 16), 0, st>>>(G, S, Dx, Dy, P,
                                                                         1.0 / ((double)G * G));
  CKL("k_psf_gemm");
  if (P_out) CK(cudaMemcpyAsync(P_out, P, (size_t)G * G * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return NLINV_OK;
}

int nlinv_grid(nlinv_plan_t pl, int S, const double* kxy, const void* y, void* Y_out, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (S <= 0 || !kxy || !y || !Y_out || ((uintptr_t)kxy & 7u) || !aligned8(y) || !aligned8(Y_out))
    return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int N = pl->N, J = pl->J;
  RC(ensure_prep(pl, (size_t)2 * S * N * sizeof(float2)));
  float2* Ex = (float2*)pl->prep;
  float2* Ey = Ex + (size_t)S * N;
  k_ndft_tables<<<(S * N + 255) / 256, 256, 0, st>>>(N, S, kxy, Ex, Ey);
  CKL("k_ndft_tables");
  k_adj_ndft<<<dim3((N + 15) / 16, (N + 15) / 16, J), dim3(16, 16), 0, st>>>(
      N, S, (const float2*)y, Ex, Ey, pl->C.s, (float)(1.0 / pl->G));
  CKL("k_adj_ndft");
  return dispatch(pl->G, [&](auto k) -> int {
    using K = decltype(k);
    Launch<K> L{pl, st};
    RC(L.row_b(ROW_IMG, nullptr, nullptr, nullptr, pl->C.s, pl->C.v));
    return L.col_c(COL_FWD, nullptr, nullptr, (float2*)Y_out, pl->C.v);
  });
}

int nlinv_apply_DF(nlinv_plan_t pl, const void* xhat, const void* dx, void* z, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!xhat || !dx || !z || !aligned8(xhat) || !aligned8(dx) || !aligned8(z)) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const float2* xh = (const float2*)xhat;
  const float2* d = (const float2*)dx;
  const size_t NN = (size_t)pl->N * pl->N;
  return dispatch(pl->G, [&](auto k) -> int {
    using K = decltype(k);
    Launch<K> L{pl, st};
    RC(L.coils(xh));
    RC(L.coil_y(d + NN, pl->C.h));
    RC(L.row_b(ROW_LIN, pl->C.h, xh, d, nullptr, pl->C.v));
    return L.col_c(COL_FWD, nullptr, nullptr, (float2*)z, pl->C.v);
  });
}

int nlinv_apply_DFH(nlinv_plan_t pl, const void* xhat, const void* z, void* dx_out, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!xhat || !z || !dx_out || !aligned8(xhat) || !aligned8(z) || !aligned8(dx_out)) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const float2* xh = (const float2*)xhat;
  return dispatch(pl->G, [&](auto k) -> int {
    using K = decltype(k);
    Launch<K> L{pl, st};
    RC(L.coils(xh));
    RC(L.col_c(COL_INV, nullptr, (const float2*)z, nullptr, pl->C.v));
    RC(L.row_d(xh, pl->C.v, pl->C.s, pl->C.kb));
    return L.col_e(E_DFH, 0.f, 0, pl->C.kb, pl->C.s, nullptr, nullptr, (float2*)dx_out, nullptr, SLOT_PQ);
  });
}

int nlinv_apply_normal(nlinv_plan_t pl, const void* xhat, const void* dx, int turn, double alpha, void* out,
                       nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!xhat || !dx || !out || !aligned8(xhat) || !aligned8(dx) || !aligned8(out)) return NLINV_EINVAL;
  if (turn < 0 || turn >= pl->U || !(alpha >= 0.0)) return NLINV_EINVAL;
  if (out == xhat || out == dx) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const float2* xh = (const float2*)xhat;
  const float2* d = (const float2*)dx;
  const size_t NN = (size_t)pl->N * pl->N;
  const float* P = pl->psf + (size_t)turn * pl->G * pl->G;
  return dispatch(pl->G, [&](auto k) -> int {
    using K = decltype(k);
    Launch<K> L{pl, st};
    RC(L.coils(xh));
    RC(L.coil_y(d + NN, pl->C.h));
    RC(L.row_b(ROW_LIN, pl->C.h, xh, d, nullptr, pl->C.v));
    RC(L.col_c(COL_TOEP, P, nullptr, nullptr, pl->C.v));
    RC(L.row_d(xh, pl->C.v, pl->C.s, pl->C.kb));
    return L.col_e(E_NORMAL, (float)alpha, 0, pl->C.kb, pl->C.s, nullptr, (float2*)d, (float2*)out, nullptr,
                   SLOT_PQ);
  });
}

int nlinv_frame(nlinv_plan_t pl, const void* Y, int turn, const void* x_prev, void* x_out, void* rho_out,
                void* img_out, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!Y || !x_out || !aligned8(Y) || !aligned8(x_out)) return NLINV_EINVAL;
  if ((x_prev && !aligned8(x_prev)) || (rho_out && !aligned8(rho_out)) || (img_out && !aligned8(img_out)))
    return NLINV_EINVAL;
  if (turn < 0 || turn >= pl->U) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const nlinv_params_t& p = pl->prm;
  FrameArgs F;
  std::memset(&F, 0, sizeof(F));
  F.io.Y = (const float2*)Y;
  F.io.P = pl->psf + (size_t)turn * pl->G * pl->G;
  F.io.xprev = (const float2*)x_prev;
  F.io.xout = (float2*)x_out;
  F.io.rho_out = (float2*)rho_out;
  F.io.img_out = (float2*)img_out;
  F.M = p.newton_steps;
  F.K = p.cg_iters;
  F.damping = (float)p.damping;
  for (int n = 0; n < F.M; ++n) F.alpha[n] = (float)(p.alpha0 * std::pow(p.q, n));
  Ctx C = pl->C;
  const int NN = pl->N * pl->N;
  return dispatch(pl->G, [&](auto k) -> int {
    using K = decltype(k);
    if (p.exec_mode == 0) {
      CK(cudaMemsetAsync(C.bar, 0, 2 * sizeof(unsigned), st));
      void* args[] = {(void*)&C, (void*)&F};
      CK(cudaLaunchCooperativeKernel((const void*)k_frame<K>, dim3(pl->coop_grid), dim3(K::BS), args,
                                     (size_t)K::SMEM, st));
      return NLINV_OK;
    }
    Launch<K> L{pl, st, pl->coop_grid};
    const int ge = plan_grid((int)((C.nx + 255) / 256), 1);
    k_init<<<ge, 256, 0, st>>>(C, F.io.xprev, F.damping);
    CKL("k_init");
    for (int n = 0; n < F.M; ++n) {
      const float alpha = F.alpha[n];
      RC(L.coil_y(C.xn + NN, C.h));
      RC(L.row_b(ROW_COIL, C.h, C.xn, nullptr, nullptr, C.v));
      RC(L.col_c(COL_RHS, F.io.P, F.io.Y, nullptr, C.v));
      RC(L.row_d(C.xn, C.v, C.s, C.kb));
      RC(L.col_e(E_RHS, alpha, 0, C.kb, C.s, nullptr, nullptr, C.rb[0], C.Hr, SLOT_RR0));
      for (int kk = 0; kk < F.K; ++kk) {
        float2* pk = C.pb[kk & 1];
        const float2* pm = C.pb[(kk + 1) & 1];
        RC(L.row_cg(kk, pm, pk, C.v));
        RC(L.col_c(COL_CG, F.io.P, nullptr, nullptr, C.v, kk));
        RC(L.row_d(C.xn, C.v, C.s, C.kb));
        RC(L.col_e(E_CG, alpha, kk, C.kb, C.s, pm, pk, C.q, nullptr, SLOT_PQ));
        RC(L.upd(kk, kk == F.K - 1, pk));
      }
    }
    RC(L.coils(C.xn));
    k_final<<<ge, 256, 0, st>>>(C, F.io.xout, F.io.rho_out, F.io.img_out);
    CKL("k_final");
    return NLINV_OK;
  });
}

int nlinv_batch(const nlinv_frame_desc_t* frames, int nframes, nlinv_stream_t stream) {
  if (!frames || nframes <= 0) return NLINV_EINVAL;
  // group the frames by plan, keeping their order
  std::vector<nlinv_plan_s*> plans;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < nframes; ++i) {
    const nlinv_frame_desc_t& d = frames[i];
    nlinv_plan_s* pl = d.plan;
    if (!pl) return NLINV_EINVAL;
    if (!d.Y || !d.x_out || !aligned8(d.Y) || !aligned8(d.x_out)) return NLINV_EINVAL;
    if ((d.x_prev && !aligned8(d.x_prev)) || (d.rho_out && !aligned8(d.rho_out)) ||
        (d.img_out && !aligned8(d.img_out)))
      return NLINV_EINVAL;
    if (d.turn < 0 || d.turn >= pl->U) return NLINV_EINVAL;
    size_t g = 0;
    while (g < plans.size() && plans[g] != pl) ++g;
    if (g == plans.size()) {
      plans.push_back(pl);
      members.emplace_back();
    }
    members[g].push_back(i);
  }
  // x_last dependencies: an earlier frame of the same plan in this call, or
  // a buffer that no frame of this call writes
  std::vector<int> dep(nframes, -1);
  for (int i = 0; i < nframes; ++i) {
    const nlinv_frame_desc_t& d = frames[i];
    if (d.x_last && !aligned8(d.x_last)) return NLINV_EINVAL;
    for (int j = 0; j < nframes; ++j) {
      if (j == i) continue;
      if (d.x_prev && d.x_prev == frames[j].x_out) return NLINV_EINVAL;
      if (d.x_last && d.x_last == frames[j].x_out) {
        if (j > i || frames[j].plan != d.plan) return NLINV_EINVAL;
        dep[i] = j;
      }
    }
  }
  double wsum = 0.0;
  std::vector<double> w(plans.size());
  for (size_t g = 0; g < plans.size(); ++g) {
    nlinv_plan_s* pl = plans[g];
    if ((int)members[g].size() > pl->max_batch) return NLINV_EINVAL;
    if (pl->dev != plans[0]->dev || pl->nsm != plans[0]->nsm) return NLINV_EINVAL;
    w[g] = (double)members[g].size() * pl->J * (double)pl->G * pl->G * std::log2((double)pl->G);
    wsum += w[g];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool fork = plans.size() > 1;
  if (fork) CK(cudaEventRecord(plans[0]->ev_fork, st));
  const int nsm = plans[0]->nsm;
  for (size_t g = 0; g < plans.size(); ++g) {
    nlinv_plan_s* pl = plans[g];
    const nlinv_params_t& p = pl->prm;
    BatchArgs B;
    std::memset(&B, 0, sizeof(B));
    B.nf = (int)members[g].size();
    B.M = p.newton_steps;
    B.K = p.cg_iters;
    B.damping = (float)p.damping;
    for (int n = 0; n < B.M; ++n) B.alpha[n] = (float)(p.alpha0 * std::pow(p.q, n));
    B.fstride = pl->fstride;
    for (int f = 0; f < B.nf; ++f) {
      const nlinv_frame_desc_t& d = frames[members[g][f]];
      B.io[f].Y = (const float2*)d.Y;
      B.io[f].P = pl->psf + (size_t)d.turn * pl->G * pl->G;
      B.io[f].xprev = (const float2*)d.x_prev;
      B.io[f].xout = (float2*)d.x_out;
      B.io[f].rho_out = (float2*)d.rho_out;
      B.io[f].img_out = (float2*)d.img_out;
      B.io[f].xlast = (const float2*)d.x_last;
    }
    for (int f = 0; f < B.nf; ++f) {   // completion flags of the frames others wait on
      const int i = members[g][f];
      if (dep[i] < 0) continue;
      int fd = 0;
      while (members[g][fd] != dep[i]) ++fd;
      B.io[fd].done = pl->C.bar + (size_t)fd * kBarStride + 1;
      B.io[f].wait = pl->C.bar + (size_t)fd * kBarStride + 1;
    }
    // this group's share of the SMs, at least one CTA per frame
    int sms = fork ? (int)std::lround(nsm * w[g] / wsum) : nsm;
    if (sms < 1) sms = 1;
    int grid = sms * pl->batch_occ;
    if (grid < B.nf) grid = B.nf;
    if (grid > pl->batch_occ * nsm) grid = pl->batch_occ * nsm;
    if (grid < B.nf) return NLINV_EINVAL;
    cudaStream_t gs = fork ? pl->aux : st;
    if (fork) CK(cudaStreamWaitEvent(gs, plans[0]->ev_fork, 0));
    Ctx C = pl->C;
    const int rc = dispatch(pl->G, [&](auto k) -> int {
      using K = decltype(k);
      CK(cudaMemsetAsync(C.bar, 0, (size_t)B.nf * kBarStride * sizeof(unsigned), gs));
      void* args[] = {(void*)&C, (void*)&B};
      CK(cudaLaunchCooperativeKernel((const void*)k_batch<K>, dim3(grid), dim3(K::BS), args,
                                     (size_t)K::SMEM, gs));
      return NLINV_OK;
    });
    if (rc != NLINV_OK) return rc;
    if (fork) {
      CK(cudaEventRecord(pl->ev_done, gs));
      CK(cudaStreamWaitEvent(st, pl->ev_done, 0));
    }
  }
  return NLINV_OK;
}

int nlinv_stream_source(int n, int delay, int warmup, int* src_out) {
  if (n < 0 || delay < 1 || warmup < 0 || !src_out) return NLINV_EINVAL;
  *src_out = n <= warmup ? n - 1 : warmup + ((n - warmup - 1) / delay) * delay;
  return NLINV_OK;
}

int nlinv_stream_schedule(int nframes, int delay, int warmup, int last_from_prev, int* group_out,
                          int* source_out, int* last_out) {
  if (nframes < 0 || delay < 1 || warmup < 0) return NLINV_EINVAL;
  int ngroups = 0;
  for (int n = 0; n < nframes; ++n) {
    // launch groups: 0, 1, ..., warmup one frame each, then runs of `delay`
    const int g = n <= warmup ? n : warmup + 1 + (n - warmup - 1) / delay;
    int src = -1;
    nlinv_stream_source(n, delay, warmup, &src);
    if (group_out) group_out[n] = g;
    if (source_out) source_out[n] = src;
    if (last_out) last_out[n] = (last_from_prev && n > 0 && src != n - 1) ? n - 1 : -1;
    ngroups = g + 1;
  }
  return ngroups;
}

int nlinv_run_streams(const nlinv_stream_desc_t* streams, int nstreams, nlinv_stream_t stream) {
  if (!streams || nstreams <= 0) return NLINV_EINVAL;
  std::vector<std::vector<int>> grp(nstreams), src(nstreams), last(nstreams);
  int ngroups = 0;
  for (int s = 0; s < nstreams; ++s) {
    const nlinv_stream_desc_t& d = streams[s];
    if (!d.plan || d.nframes < 0) return NLINV_EINVAL;
    if (d.nframes > 0 && (!d.Y || !d.turns || !d.x_out)) return NLINV_EINVAL;
    if (d.delay > d.plan->max_batch) return NLINV_EINVAL;
    for (int t = 0; t < s; ++t)
      if (streams[t].plan == d.plan) return NLINV_EINVAL;
    grp[s].resize(d.nframes);
    src[s].resize(d.nframes);
    last[s].resize(d.nframes);
    const int ng = nlinv_stream_schedule(d.nframes, d.delay, d.warmup, d.last_from_prev, grp[s].data(),
                                         src[s].data(), last[s].data());
    if (ng < 0) return ng;
    if (ng > ngroups) ngroups = ng;
  }
  std::vector<nlinv_frame_desc_t> fr;
  for (int g = 0; g < ngroups; ++g) {
    fr.clear();
    for (int s = 0; s < nstreams; ++s) {
      const nlinv_stream_desc_t& d = streams[s];
      for (int n = 0; n < d.nframes; ++n) {
        if (grp[s][n] != g) continue;
        nlinv_frame_desc_t f;
        std::memset(&f, 0, sizeof(f));
        f.plan = d.plan;
        f.Y = d.Y[n];
        f.turn = d.turns[n];
        f.x_prev = src[s][n] < 0 ? d.x_init : d.x_out[src[s][n]];
        f.x_out = d.x_out[n];
        f.img_out = d.img_out ? d.img_out[n] : nullptr;
        f.x_last = last[s][n] >= 0 ? d.x_out[last[s][n]] : nullptr;
        fr.push_back(f);
      }
    }
    if (!fr.empty()) RC(nlinv_batch(fr.data(), (int)fr.size(), stream));
  }
  return NLINV_OK;
}

int nlinv_sync(nlinv_plan_t pl, nlinv_stream_t stream) {
  RC(check_plan(pl));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  int h = 0;
  CK(cudaMemcpy(&h, pl->C.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) CK(cudaMemset(pl->C.err, 0, sizeof(int)));
  return h;
}

int nlinv_wait_flag(nlinv_plan_t pl, const int* flag, int expected, long long spin_limit, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!flag || spin_limit <= 0 || ((uintptr_t)flag & 3u)) return NLINV_EINVAL;
  k_wait_flag<<<1, 32, 0, (cudaStream_t)stream>>>(flag, expected, spin_limit, pl->C.err);
  CKL("k_wait_flag");
  return NLINV_OK;
}

}  // extern "C"

// ======================================================================
// Allocation-free normal operator.
//
// Some callers cannot call cudaMalloc: a reconstruction loop that must not
// allocate (or implicitly synchronise the device) once it is running, or a
// host framework that hands out all device memory from its own pools.  For
// them nlinv_apply_normal_static runs the same phase kernels as
// nlinv_apply_normal with every intermediate in one file-scope __device__
// array that is part of the loaded module, so no call allocates.
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[64] = {};
// the (G, Gc, w_a, w_l) whose twiddle and D_W^-1 tables the array holds, per
// device: a call with the same sizes and weight constants skips the table
// kernel (the tables stay valid until a call with other values rewrites them)
struct StaticKey {
  int G = 0, Gc = 0;
  double w_a = 0.0, w_l = 0.0;
};
StaticKey g_static_key[64];

// twiddles w_G^k and the D_W^-1 table, computed on the device in FP64
__global__ void k_static_tables(int G, int Gc, double w_a, double w_l, float2* tw, float* dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < G) {
    double sn, cs;
    sincospi(-2.0 * (double)i / G, &sn, &cs);
    tw[i] = make_float2((float)cs, (float)sn);
  }
  if (i < Gc * Gc) {
    const int iy = i / Gc, ix = i - iy * Gc;
    const int fy = iy < (Gc + 1) / 2 ? iy : iy - Gc;
    const int fx = ix < (Gc + 1) / 2 ? ix : ix - Gc;
    const double ky = 2.0 * fy / G, kx = 2.0 * fx / G;
    dinv[i] = (float)pow(1.0 + w_a * (kx * kx + ky * ky), -w_l / 2.0);
  }
}

// set-up once per device (with that device current): the device address of
// the scratch array and the constant twiddle table.  *fresh is set when the
// array's tables do not hold (G, Gc, w_a, w_l); static_tables_written()
// records them once the table kernel is enqueued.
int static_scratch(void** out, int G, int Gc, double w_a, double w_l, bool* fresh) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return NLINV_EINVAL;
  RC(ensure_constants(dev));
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_ptr[dev] = p;
  }
  const StaticKey& k = g_static_key[dev];
  *fresh = !(k.G == G && k.Gc == Gc && k.w_a == w_a && k.w_l == w_l);
  *out = g_static_ptr[dev];
  return NLINV_OK;
}

void static_tables_written(int G, int Gc, double w_a, double w_l) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticKey& k = g_static_key[dev];
  k.G = G;
  k.Gc = Gc;
  k.w_a = w_a;
  k.w_l = w_l;
}

}  // namespace

extern "C" int nlinv_apply_normal_static(int N, int J, int Gc, double w_a, double w_l, const void* xhat,
                                         const void* dx, const float* psf, double alpha, void* out,
                                         nlinv_stream_t stream) {
  const int G = 2 * N;
  if (N <= 0 || J <= 0 || J > 4096) return NLINV_EINVAL;
  if (!supported_grid(G)) return NLINV_EUNSUPPORTED;
  if (Gc == 0) Gc = G / 4;
  if (Gc < 2 || Gc > G || (Gc & 1)) return NLINV_EINVAL;
  if (!(alpha >= 0.0) || !(w_a >= 0.0) || !(w_l >= 0.0)) return NLINV_EINVAL;
  if (!xhat || !dx || !psf || !out || !aligned8(xhat) || !aligned8(dx) || !aligned8(out) ||
      ((uintptr_t)psf & 3u))
    return NLINV_EINVAL;
  if (out == xhat || out == dx) return NLINV_EINVAL;
  // scratch layout: tw, dinv, c, h, v, s, kb, partials, counters
  const size_t f2 = sizeof(float2);
  size_t off[12];
  size_t tot = 0;
  int nb = 0;
  auto take = [&](size_t bytes) {
    off[nb++] = tot;
    tot += align_up(bytes);
  };
  take(G * f2);
  take((size_t)Gc * Gc * sizeof(float));
  take((size_t)J * N * N * f2);
  take((size_t)J * N * Gc * f2);
  take((size_t)J * N * G * f2);
  take((size_t)J * N * N * f2);
  take((size_t)J * N * Gc * f2);
  take((size_t)NSLOT * kMaxPart * sizeof(float2));
  take(sizeof(int) + 2 * sizeof(unsigned));
  if (tot > kStaticScratchBytes) return NLINV_EINVAL;
  void* base_v = nullptr;
  bool fresh = true;
  RC(static_scratch(&base_v, G, Gc, w_a, w_l, &fresh));
  char* base = (char*)base_v;
  cudaStream_t st = (cudaStream_t)stream;

  nlinv_plan_s tmp;
  Ctx& C = tmp.C;
  std::memset(&C, 0, sizeof(C));
  C.N = N;
  C.G = G;
  C.Gc = Gc;
  C.J = J;
  C.nx = N * N + J * Gc * Gc;
  C.U = 1;
  C.inv_G = (float)(1.0 / G);
  C.inv_G2 = (float)(1.0 / ((double)G * G));
  float2* tw = (float2*)(base + off[0]);
  float* dinv = (float*)(base + off[1]);
  C.tw = tw;
  C.dinv = dinv;
  C.psf = psf;
  C.c = (float2*)(base + off[2]);
  C.h = (float2*)(base + off[3]);
  C.v = (float2*)(base + off[4]);
  C.s = (float2*)(base + off[5]);
  C.kb = (float2*)(base + off[6]);
  C.part = (float2*)(base + off[7]);
  C.err = (int*)(base + off[8]);
  C.bar = (unsigned*)(C.err + 1);
  C.spin_limit = 1LL << 22;
  if (fresh) {
    const int nt = (G > Gc * Gc ? G : Gc * Gc);
    k_static_tables<<<(nt + 255) / 256, 256, 0, st>>>(G, Gc, w_a, w_l, tw, dinv);
    CKL("k_static_tables");
    static_tables_written(G, Gc, w_a, w_l);
  }
  const float2* xh = (const float2*)xhat;
  const float2* d = (const float2*)dx;
  const size_t NN = (size_t)N * N;
  return dispatch(G, [&](auto k) -> int {
    using K = decltype(k);
    RC(set_smem_attrs<K>());
    Launch<K> L{&tmp, st};
    RC(L.coils(xh));
    RC(L.coil_y(d + NN, C.h));
    RC(L.row_b(ROW_LIN, C.h, xh, d, nullptr, C.v));
    RC(L.col_c(COL_TOEP, psf, nullptr, nullptr, C.v));
    RC(L.row_d(xh, C.v, C.s, C.kb));
    return L.col_e(E_NORMAL, (float)alpha, 0, C.kb, C.s, nullptr, (float2*)d, (float2*)out, nullptr, SLOT_PQ);
  });
}

// ======================================================================
// Reverse-mode derivative of one frame through the unrolled IRGNM / CG
// (Sec. 2.2, Eqs. (2)-(5)).  F^ is bilinear with the symmetric form
// B(x, d) = DF(x)[d], so every derivative is DF / DF^H at some
// linearisation point:
//   A(x) p = DF(x)^H P DF(x) p + alpha p
//     -> x-bar += DF(qbar)^H P DF(x) p + DF(p)^H P DF(x) qbar
//   b(x) = DF(x)^H z - alpha (x - x_ref),  z = Y - P F^(x),  F^(x) = B(x, x) / 2
//     -> x-bar += DF(bbar)^H z - DF(x)^H P DF(x) bbar - alpha bbar
//        Y-bar += DF(x) bbar,  alpha-bar -= <bbar, x - x_ref>_R,  x_ref-bar += alpha bbar
// The CG of each Newton step is recomputed from its checkpoint x^_n and
// reversed step by step; scalars are handled on the host in FP64.
namespace {

// y = a x + b y  (a as a float pair; b == 0 overwrites y)
__global__ void k_axpby(long long n, float2* y, const float2* x, float ahi, float alo, float b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 xv = x[i];
    float2 base = make_float2(0.f, 0.f);
    if (b != 0.f) {
      const float2 yv = y[i];
      base = make_float2(b * yv.x, b * yv.y);
    }
    y[i] = make_float2(fmaf(ahi, xv.x, fmaf(alo, xv.x, base.x)), fmaf(ahi, xv.y, fmaf(alo, xv.y, base.y)));
  }
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;   // valid in lane 0
}

// per-block FP64 partials of Re <u, v>
__global__ void k_dot_part(long long n, const float2* u, const float2* v, double* part) {
  __shared__ double sw[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 a = u[i], b = v[i];
    acc = fma((double)a.x, (double)b.x, fma((double)a.y, (double)b.y, acc));
  }
  acc = warp_sum_f64(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sw[w];
    part[blockIdx.x] = a;
  }
}

// one warp: lane l adds partials l, l + 32, ... (all loads issued first),
// then a fixed shuffle tree (a single thread adding them in turn spent
// ~19 us per call on dependent FP64 adds and loads)
__global__ void k_dot_final(int np, const double* part, double* out) {
  const int l = threadIdx.x;
  double a = 0.0;
  for (int base = 0; base < np; base += 32 * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * 32 + l;
      v[u] = i < np ? part[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) a += v[u];
  }
  a = warp_sum_f64(a);
  if (l == 0) *out = a;
}

// several Re<u_j, v_j> in one pass over n elements (per-block FP64 partials,
// [MD][kDotBlocks]), reduced per product by one warp each in k_dots_final
constexpr int kMaxDots = 8;
struct DotSet {
  const float2* u[kMaxDots];
  const float2* v[kMaxDots];
};
template <int MD>
__global__ void k_dots_part(long long n, DotSet S, double* part) {
  __shared__ double sw[MD][32];
  double acc[MD];
#pragma unroll
  for (int j = 0; j < MD; ++j) acc[j] = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < MD; ++j) {
      const float2 a = S.u[j][i], b = S.v[j][i];
      acc[j] = fma((double)a.x, (double)b.x, fma((double)a.y, (double)b.y, acc[j]));
    }
  }
#pragma unroll
  for (int j = 0; j < MD; ++j) {
    const double v = warp_sum_f64(acc[j]);
    if ((threadIdx.x & 31) == 0) sw[j][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < MD) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sw[threadIdx.x][w];
    part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = a;
  }
}
__global__ void k_dots_final(int np, const double* part, double* out) {
  const int l = threadIdx.x;
  const double* src = part + (size_t)blockIdx.x * np;
  double a = 0.0;
  for (int base = 0; base < np; base += 32 * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * 32 + l;
      v[u] = i < np ? src[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) a += v[u];
  }
  a = warp_sum_f64(a);
  if (l == 0) out[blockIdx.x] = a;
}

// z <- s P z on [J][G][G]
__global__ void k_psf_scale(int J, int G, float2* z, const float* __restrict__ P, float s) {
  const long long n = (long long)J * G * G, g2 = (long long)G * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = cscale(z[i], s * P[i % g2]);
}

// z <- Y - s P z
__global__ void k_resid(int J, int G, float2* z, const float2* __restrict__ Y, const float* __restrict__ P, float s) {
  const long long n = (long long)J * G * G, g2 = (long long)G * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float pk = s * P[i % g2];
    const float2 zv = z[i], yv = Y[i];
    z[i] = make_float2(fmaf(-pk, zv.x, yv.x), fmaf(-pk, zv.y, yv.y));
  }
}

__global__ void k_init_x(int nx, int NN, float2* x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x)
    x[i] = make_float2(i < NN ? 1.f : 0.f, 0.f);
}

constexpr int kDotBlocks = 256;

struct GradOps {
  nlinv_plan_s* pl;
  cudaStream_t st;
  const float* P;
  long long nx, nk;
  double* part;   // [kMaxDots][kDotBlocks]
  double* dres;   // device scalars [kMaxDots]
  // The plan's coil-map buffer holds W^-1 of lin's coil part when
  // coils_at == lin.  lin is the Newton step's checkpoint x^_n, which is not
  // written while it is the linearisation point; maps of any other point
  // (a buffer that may change between calls) are never reused.
  const float2* lin = nullptr;
  mutable const float2* coils_at = nullptr;
  template <class Lc>
  int coils(const Lc& L, const float2* w) const {
    if (w != nullptr && w == lin && coils_at == lin) return NLINV_OK;
    coils_at = (w == lin) ? lin : nullptr;
    return L.coils(w);
  }

  int grid(long long n) const {
    long long g = (n + 255) / 256;
    return (int)(g > 1024 ? 1024 : (g < 1 ? 1 : g));
  }
  int axpby(float2* y, const float2* x, double a, double b, long long n) const {
    const float hi = (float)a, lo = (float)(a - (double)hi);
    k_axpby<<<grid(n), 256, 0, st>>>(n, y, x, hi, lo, (float)b);
    CKL("k_axpby");
    return NLINV_OK;
  }
  int copy(float2* y, const float2* x, long long n) const {
    CK(cudaMemcpyAsync(y, x, (size_t)n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    return NLINV_OK;
  }
  int zero(float2* y, long long n) const {
    CK(cudaMemsetAsync(y, 0, (size_t)n * sizeof(float2), st));
    return NLINV_OK;
  }
  int dot(const float2* u, const float2* v, long long n, double* out) const {
    k_dot_part<<<kDotBlocks, 256, 0, st>>>(n, u, v, part);
    CKL("k_dot_part");
    k_dot_final<<<1, 32, 0, st>>>(kDotBlocks, part, dres);
    CKL("k_dot_final");
    CK(cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return NLINV_OK;
  }
  // kMaxDots products Re<u_j, v_j> with one read-back
  int dots(const DotSet& S, double* out) const {
    k_dots_part<kMaxDots><<<kDotBlocks, 256, 0, st>>>(nx, S, part);
    CKL("k_dots_part");
    k_dots_final<<<kMaxDots, 32, 0, st>>>(kDotBlocks, part, dres);
    CKL("k_dots_final");
    CK(cudaMemcpyAsync(out, dres, kMaxDots * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return NLINV_OK;
  }
  // z = DF(x)[d]
  int DF(const float2* x, const float2* d, float2* z) const {
    const size_t NN = (size_t)pl->N * pl->N;
    return dispatch(pl->G, [&](auto k) -> int {
      using K = decltype(k);
      Launch<K> L{pl, st};
      RC(coils(L, x));
      RC(L.coil_y(d + NN, pl->C.h));
      RC(L.row_b(ROW_LIN, pl->C.h, x, d, nullptr, pl->C.v));
      return L.col_c(COL_FWD, nullptr, nullptr, z, pl->C.v);
    });
  }
  // out = DF(w)^H z
  int DFH(const float2* w, const float2* z, float2* out) const {
    return dispatch(pl->G, [&](auto k) -> int {
      using K = decltype(k);
      Launch<K> L{pl, st};
      RC(coils(L, w));
      RC(L.col_c(COL_INV, nullptr, z, nullptr, pl->C.v));
      RC(L.row_d(w, pl->C.v, pl->C.s, pl->C.kb));
      return L.col_e(E_DFH, 0.f, 0, pl->C.kb, pl->C.s, nullptr, nullptr, out, nullptr, SLOT_PQ);
    });
  }
  // out = (DF(x)^H P DF(x) + alpha) d
  int normal(const float2* x, const float2* d, double alpha, float2* out) const {
    const size_t NN = (size_t)pl->N * pl->N;
    return dispatch(pl->G, [&](auto k) -> int {
      using K = decltype(k);
      Launch<K> L{pl, st};
      RC(coils(L, x));
      RC(L.coil_y(d + NN, pl->C.h));
      RC(L.row_b(ROW_LIN, pl->C.h, x, d, nullptr, pl->C.v));
      RC(L.col_c(COL_TOEP, P, nullptr, nullptr, pl->C.v));
      RC(L.row_d(x, pl->C.v, pl->C.s, pl->C.kb));
      return L.col_e(E_NORMAL, (float)alpha, 0, pl->C.kb, pl->C.s, nullptr, (float2*)d, out, nullptr, SLOT_PQ);
    });
  }
  int psf(float2* z, float s) const {
    k_psf_scale<<<grid(nk), 256, 0, st>>>(pl->J, pl->G, z, P, s);
    CKL("k_psf_scale");
    return NLINV_OK;
  }
  int resid(float2* z, const float2* Y) const {   // z <- Y - P z / 2
    k_resid<<<grid(nk), 256, 0, st>>>(pl->J, pl->G, z, Y, P, 0.5f);
    CKL("k_resid");
    return NLINV_OK;
  }
};

struct GradWS {
  float2 *ck, *b, *z, *zt, *zt2, *tp, *tq, *tr, *xb, *xbn, *pbar, *rbar, *qbar, *pb, *t1, *xref, *xrefbar, *xcg;
  double *part, *dres;
};

int grad_workspace(nlinv_plan_s* pl, GradWS& w) {
  const int M = pl->prm.newton_steps, Kc = pl->prm.cg_iters;
  const size_t nx = (size_t)pl->nx, nk = (size_t)pl->J * pl->G * pl->G;
  const size_t vb = align_up(nx * sizeof(float2)), kb = align_up(nk * sizeof(float2));
  const size_t need = vb * ((M + 1) + 1 + Kc + Kc + (Kc + 1) + 10) + 3 * kb +
                      align_up((size_t)kMaxDots * (kDotBlocks + 1) * sizeof(double));
  RC(ensure_prep(pl, need));
  char* p = (char*)pl->prep;
  auto vec = [&](size_t count) {
    float2* r = (float2*)p;
    p += vb * count;
    return r;
  };
  w.ck = vec(M + 1);
  w.b = vec(1);
  w.tp = vec(Kc > 0 ? Kc : 1);
  w.tq = vec(Kc > 0 ? Kc : 1);
  w.tr = vec(Kc + 1);
  w.xb = vec(1);
  w.xbn = vec(1);
  w.pbar = vec(1);
  w.rbar = vec(1);
  w.qbar = vec(1);
  w.pb = vec(1);
  w.t1 = vec(1);
  w.xref = vec(1);
  w.xrefbar = vec(1);
  w.xcg = vec(1);
  w.z = (float2*)p;
  p += kb;
  w.zt = (float2*)p;
  p += kb;
  w.zt2 = (float2*)p;
  p += kb;
  w.part = (double*)p;
  w.dres = w.part + (size_t)kMaxDots * kDotBlocks;
  return NLINV_OK;
}

struct CgTape {
  int K = 0;
  std::vector<double> a, beta, gamma, rho;
};

// b = DF(x)^H (Y - P F^(x)) - alpha (x - xref); leaves the residual in w.z
int grad_rhs(const GradOps& O, const GradWS& w, const float2* Y, const float2* x, double alpha, float2* b) {
  RC(O.DF(x, x, w.z));
  RC(O.resid(w.z, Y));
  RC(O.DFH(x, w.z, b));
  RC(O.axpby(b, x, -alpha, 1.0, O.nx));
  return O.axpby(b, w.xref, alpha, 1.0, O.nx);
}

// CG from zero recording p_k, q_k, r_k (k = 0..) and the scalars; delta in w.xcg
int grad_cg(const GradOps& O, const GradWS& w, const float2* x, double alpha, const float2* b, int iters,
            CgTape& T) {
  const long long nx = O.nx;
  T = CgTape();
  float2* r0 = w.tr;
  RC(O.copy(r0, b, nx));
  RC(O.zero(w.xcg, nx));
  double rr = 0.0;
  RC(O.dot(r0, r0, nx, &rr));
  T.rho.push_back(rr);
  if (iters > 0) RC(O.copy(w.tp, r0, nx));
  for (int k = 0; k < iters; ++k) {
    if (rr == 0.0) break;
    float2* p = w.tp + (size_t)k * (size_t)nx;
    float2* q = w.tq + (size_t)k * (size_t)nx;
    float2* r = w.tr + (size_t)k * (size_t)nx;
    float2* r1 = w.tr + (size_t)(k + 1) * (size_t)nx;
    RC(O.normal(x, p, alpha, q));
    double pq = 0.0;
    RC(O.dot(p, q, nx, &pq));
    if (!(pq > 0.0) || !std::isfinite(pq)) return NLINV_ENUMERIC;
    const double a = rr / pq;
    RC(O.axpby(w.xcg, p, a, 1.0, nx));
    RC(O.copy(r1, r, nx));
    RC(O.axpby(r1, q, -a, 1.0, nx));
    double rn = 0.0;
    RC(O.dot(r1, r1, nx, &rn));
    const double beta = rn / rr;
    T.a.push_back(a);
    T.gamma.push_back(pq);
    T.beta.push_back(beta);
    T.rho.push_back(rn);
    T.K = k + 1;
    if (k + 1 < iters) {
      float2* p1 = w.tp + (size_t)(k + 1) * (size_t)nx;
      RC(O.copy(p1, r1, nx));
      RC(O.axpby(p1, p, beta, 1.0, nx));
    }
    rr = rn;
  }
  return NLINV_OK;
}

}  // namespace

extern "C" int nlinv_set_alpha0(nlinv_plan_t pl, double alpha0) {
  if (!pl || !(alpha0 > 0.0)) return NLINV_EINVAL;
  pl->prm.alpha0 = alpha0;
  return NLINV_OK;
}

extern "C" int nlinv_frame_vjp(nlinv_plan_t pl, const void* Y, int turn, const void* x_prev, const void* gbar,
                               void* Ybar_out, double* alpha0_bar_out, void* xprev_bar_out,
                               nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!Y || !gbar || !Ybar_out || !aligned8(Y) || !aligned8(gbar) || !aligned8(Ybar_out)) return NLINV_EINVAL;
  if ((x_prev && !aligned8(x_prev)) || (xprev_bar_out && !aligned8(xprev_bar_out))) return NLINV_EINVAL;
  if (turn < 0 || turn >= pl->U) return NLINV_EINVAL;
  const nlinv_params_t& prm = pl->prm;
  const int M = prm.newton_steps, Kc = prm.cg_iters;
  GradWS w;
  RC(grad_workspace(pl, w));
  GradOps O{pl, (cudaStream_t)stream, pl->psf + (size_t)turn * pl->G * pl->G, pl->nx,
            (long long)pl->J * pl->G * pl->G, w.part, w.dres};
  const long long nx = O.nx, nk = O.nk;
  const float2* Yd = (const float2*)Y;
  // x^_0 and x_ref
  if (x_prev) {
    RC(O.copy(w.ck, (const float2*)x_prev, nx));
  } else {
    k_init_x<<<O.grid(nx), 256, 0, O.st>>>((int)nx, pl->N * pl->N, w.ck);
    CKL("k_init_x");
  }
  RC(O.copy(w.xref, w.ck, nx));
  RC(O.axpby(w.xref, w.xref, 0.0, prm.damping, nx));
  // forward: checkpoints x^_n
  CgTape T;
  for (int n = 0; n < M; ++n) {
    const float2* x = w.ck + (size_t)n * (size_t)nx;
    float2* x1 = w.ck + (size_t)(n + 1) * (size_t)nx;
    const double alpha = prm.alpha0 * std::pow(prm.q, n);
    O.lin = x;
    RC(grad_rhs(O, w, Yd, x, alpha, w.b));
    RC(grad_cg(O, w, x, alpha, w.b, Kc, T));
    RC(O.copy(x1, x, nx));
    RC(O.axpby(x1, w.xcg, 1.0, 1.0, nx));
  }
  // reverse
  float2* Ybar = (float2*)Ybar_out;
  RC(O.zero(Ybar, nk));
  RC(O.zero(w.xrefbar, nx));
  RC(O.copy(w.xb, (const float2*)gbar, nx));
  double a0bar = 0.0;
  for (int n = M - 1; n >= 0; --n) {
    const float2* x = w.ck + (size_t)n * (size_t)nx;
    const double alpha = prm.alpha0 * std::pow(prm.q, n);
    O.lin = x;
    RC(grad_rhs(O, w, Yd, x, alpha, w.b));            // residual z stays in w.z
    RC(grad_cg(O, w, x, alpha, w.b, Kc, T));
    double alpha_bar = 0.0;
    RC(O.copy(w.xbn, w.xb, nx));                      // x^_{n+1} = x^_n + delta
    RC(O.zero(w.pbar, nx));
    RC(O.zero(w.rbar, nx));
    std::vector<double> rhobar(T.K + 1, 0.0);
    for (int k = T.K - 1; k >= 0; --k) {
      const float2* p = w.tp + (size_t)k * (size_t)nx;
      const float2* q = w.tq + (size_t)k * (size_t)nx;
      const float2* r1 = w.tr + (size_t)(k + 1) * (size_t)nx;
      const double a = T.a[k], beta = T.beta[k], gamma = T.gamma[k];
      const double rk = T.rho[k], rk1 = T.rho[k + 1];
      // every inner product this step needs, from the vectors as they enter
      // it (the updates below are linear in them): one read-back per step
      //   D0 <p, pbar>  D1 <q, rbar>  D2 <q, pbar>  D3 <q, r1>
      //   D4 <p, xb>    D5 <p, rbar>  D6 <p, r1>    D7 <p, p>
      DotSet S;
      const float2* U[kMaxDots] = {p, q, q, q, p, p, p, p};
      const float2* V[kMaxDots] = {w.pbar, w.rbar, w.pbar, r1, w.xb, w.rbar, r1, p};
      for (int j = 0; j < kMaxDots; ++j) {
        S.u[j] = U[j];
        S.v[j] = V[j];
      }
      double D[kMaxDots];
      RC(O.dots(S, D));
      RC(O.axpby(w.rbar, w.pbar, 1.0, 1.0, nx));      // p_{k+1} = r_{k+1} + beta p_k
      const double betabar = D[0];
      RC(O.copy(w.pb, w.pbar, nx));
      RC(O.axpby(w.pb, w.pb, 0.0, beta, nx));
      rhobar[k + 1] += betabar / rk;                  // beta = rho_{k+1} / rho_k
      rhobar[k] -= betabar * rk1 / (rk * rk);
      const double c = 2.0 * rhobar[k + 1];
      RC(O.axpby(w.rbar, r1, c, 1.0, nx));            // rho_{k+1} = <r, r>
      double abar = -(D[1] + D[2] + c * D[3]);        // r_{k+1} = r_k - a q_k
      RC(O.copy(w.qbar, w.rbar, nx));
      RC(O.axpby(w.qbar, w.qbar, 0.0, -a, nx));
      abar += D[4];                                   // x_{k+1} = x_k + a p_k
      RC(O.axpby(w.pb, w.xb, a, 1.0, nx));
      rhobar[k] += abar / gamma;                      // a = rho_k / gamma_k
      const double gammabar = -abar * rk / (gamma * gamma);
      RC(O.axpby(w.pb, q, gammabar, 1.0, nx));        // gamma = <p, q>
      RC(O.axpby(w.qbar, p, gammabar, 1.0, nx));
      RC(O.normal(x, w.qbar, alpha, w.t1));           // q = A p
      RC(O.axpby(w.pb, w.t1, 1.0, 1.0, nx));
      // A depends on alpha and x^_n: <p, qbar>, qbar = -a rbar' + gammabar p
      alpha_bar += -a * (D[5] + D[0] + c * D[6]) + gammabar * D[7];
      // both DF at x^_n first, while its coil maps are current
      RC(O.DF(x, p, w.zt));
      RC(O.psf(w.zt, 1.f));
      RC(O.DF(x, w.qbar, w.zt2));
      RC(O.psf(w.zt2, 1.f));
      RC(O.DFH(w.qbar, w.zt, w.t1));
      RC(O.axpby(w.xbn, w.t1, 1.0, 1.0, nx));
      RC(O.DFH(p, w.zt2, w.t1));
      RC(O.axpby(w.xbn, w.t1, 1.0, 1.0, nx));
      std::swap(w.pbar, w.pb);
    }
    // p_0 = r_0 = b, rho_0 = <r_0, r_0>:  b-bar
    RC(O.axpby(w.rbar, w.pbar, 1.0, 1.0, nx));
    RC(O.axpby(w.rbar, w.tr, 2.0 * rhobar[0], 1.0, nx));
    const float2* bbar = w.rbar;
    // right-hand side
    RC(O.DFH(bbar, w.z, w.t1));
    RC(O.axpby(w.xbn, w.t1, 1.0, 1.0, nx));
    RC(O.DF(x, bbar, w.zt));
    {  // Y-bar += DF(x) b-bar
      const float hi = 1.f;
      k_axpby<<<O.grid(nk), 256, 0, O.st>>>(nk, Ybar, w.zt, hi, 0.f, 1.f);
      CKL("k_axpby");
    }
    RC(O.psf(w.zt, 1.f));
    RC(O.DFH(x, w.zt, w.t1));
    RC(O.axpby(w.xbn, w.t1, -1.0, 1.0, nx));
    RC(O.axpby(w.xbn, bbar, -alpha, 1.0, nx));
    double t1 = 0.0, t2 = 0.0;
    RC(O.dot(bbar, x, nx, &t1));
    RC(O.dot(bbar, w.xref, nx, &t2));
    alpha_bar -= (t1 - t2);
    a0bar += std::pow(prm.q, n) * alpha_bar;
    RC(O.axpby(w.xrefbar, bbar, alpha, 1.0, nx));
    std::swap(w.xb, w.xbn);
  }
  if (alpha0_bar_out) *alpha0_bar_out = a0bar;
  if (xprev_bar_out) {
    if (x_prev) {
      RC(O.copy((float2*)xprev_bar_out, w.xb, nx));
      RC(O.axpby((float2*)xprev_bar_out, w.xrefbar, prm.damping, 1.0, nx));
    } else {
      RC(O.zero((float2*)xprev_bar_out, nx));
    }
  }
  CK(cudaStreamSynchronize(O.st));
  return NLINV_OK;
}

#ifdef NLINV_TIMELINE
extern "C" int nlinv_debug_timeline(unsigned long long* host, int n) {
  if (n > 160 * 1024) n = 160 * 1024;
  CK(cudaMemcpyFromSymbol(host, g_timeline, (size_t)n * sizeof(unsigned long long)));
  return NLINV_OK;
}
extern "C" int nlinv_debug_stages(unsigned long long* ns, unsigned long long* cnt) {
  CK(cudaMemcpyFromSymbol(ns, nlinv::g_stage_ns, sizeof(unsigned long long) * 64));
  CK(cudaMemcpyFromSymbol(cnt, nlinv::g_stage_n, sizeof(unsigned long long) * 64));
  return NLINV_OK;
}
#endif
