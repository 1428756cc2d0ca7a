// Kernels of the NLINV hot path for one FFT grid size and the host
// operations that launch them (the GridOps table of common.h).  grid.cu
// includes this once per compiled grid size, so each size is its own
// translation unit: the fused phase kernels (one launch per phase), the
// persistent grid kernel k_frame, the cluster kernel k_frame_cl and the
// batch kernel k_batch (Sec. 2.2, Eqs. (2)-(5); Sec. 3.3).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.h"
#include "phases_cgr.cuh"

// CTAs per SM the frame-indexed phase kernels (kf_*) are compiled for (caps
// their registers; one measured fastest at the 320 grid: two cost 34 % per
// frame in register spills)
#ifndef NLINV_PMINB
#define NLINV_PMINB 1
#endif

namespace nlinv {
namespace {

// ---------------------------------------------------- kernel wrappers
// every CTA of a one-frame launch works on that frame
__device__ __forceinline__ Ctx whole_grid(const Ctx& C0) {
  Ctx C = C0;
  C.bid = blockIdx.x;
  C.nb = gridDim.x;
  return C;
}

// Entry of a one-phase kernel: let the next kernel of the stream be launched
// (programmatic dependent launch: its CTAs take SMs as ours leave), then wait
// until the previous kernel has finished and its stores are visible.  Both
// are no-ops for a kernel launched without programmatic dependencies.
__device__ __forceinline__ Ctx phase_entry(const Ctx& C0) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  return whole_grid(C0);
}

template <class K>
__global__ void __launch_bounds__(K::BS, K::OMINB) k_coil_y(Ctx C0, const float2* src, float2* hout) {
  const Ctx C = phase_entry(C0);
  extern __shared__ float2 sm[];
  phase_coil_y<K>(C, sm, src, hout);
}

template <class K>
__global__ void __launch_bounds__(K::BS, K::OMINB) k_row_b(Ctx C0, int mode, const float2* hin, const float2* rho,
                                                 const float2* drho, const float2* img, float2* vout) {
  const Ctx C = phase_entry(C0);
  extern __shared__ float2 sm[];
  phase_row_b<K>(C, sm, mode, hin, rho, drho, img, vout);
}

template <class K>
__global__ void __launch_bounds__(K::BS, K::OMINB) k_row_deapod(Ctx C0, const float* dap, float scale, float2* v) {
  const Ctx C = phase_entry(C0);
  extern __shared__ float2 sm[];
  phase_row_deapod<K>(C, sm, dap, scale, v);
}

// the operator column passes, one kernel per mode (each compiles for its own
// operands: at two CTAs per SM the register cap otherwise spills the modes
// that need fewer)
template <class K, int MODE>
__global__ void __launch_bounds__(K::BS, K::OMINB) k_col_c(Ctx C0, const float* P, const float2* Yin,
                                                           float2* zout, float2* vio, int k) {
  const Ctx C = phase_entry(C0);
  extern __shared__ float2 sm[];
  phase_col_c<K>(C, sm, MODE, P, Yin, zout, vio, k);
}

template <class K>
__global__ void __launch_bounds__(K::BS, K::OMINB) k_row_d(Ctx C0, const float2* rho, const float2* win, float2* sout,
                                                 float2* kbout) {
  const Ctx C = phase_entry(C0);
  extern __shared__ float2 sm[];
  phase_row_d<K>(C, sm, rho, win, sout, kbout);
}

template <class K, int MODE>
__global__ void __launch_bounds__(K::BS, K::OMINB) k_col_e(Ctx C0, float alpha, int k, const float2* kbin,
                                                           const float2* sin, const float2* p_old, float2* p_new,
                                                           float2* out, float2* hout, int slot) {
  const Ctx C = phase_entry(C0);
  extern __shared__ float2 sm[];
  __shared__ float2 sred[32];
  phase_col_e<K, MODE>(C, sm, sred, alpha, k, kbin, sin, p_old, p_new, out, hout, slot);
}

// ------------------------------------------ frame-indexed phase kernels
// The per-phase path launches each phase of the IRGNM / CG once for nf frames
// of one plan: CTA b works on frame f = b / nbf as CTA b % nbf of nbf, on
// frame f's workspace (frame_ctx), so every frame sees the same CTA count in
// every phase and its CG partial sums line up.  The frames' inputs and
// outputs come from a device table written before the sequence (k_set_io),
// so one captured sequence serves every call with the same frame count.
struct PhaseBatch {
  size_t fstride;       // bytes between the frames' workspaces
  int nbf;              // CTAs per frame
  const FrameIO* io;    // device [nf]
};

__device__ __forceinline__ Ctx frame_entry(const Ctx& C0, const PhaseBatch& B, int& f) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  f = (int)(blockIdx.x / (unsigned)B.nbf);
  Ctx C = frame_ctx(C0, (size_t)f * B.fstride);
  C.bid = (int)blockIdx.x - f * B.nbf;
  C.nb = B.nbf;
  return C;
}

struct IOTable {
  FrameIO io[kMaxBatch];
};
__global__ void k_set_io(IOTable T, int nf, FrameIO* dst) {
  const int f = threadIdx.x;
  if (f < nf) dst[f] = T.io[f];
}

// x^_0 = x_prev (or rho = 1, c^ = 0), x_ref = damping x_prev
__global__ void kf_init(Ctx C0, PhaseBatch B, float damping) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  phase_init(C, B.io[f].xprev, damping);
}

// the coil part of x^_n through W^-1 along y
template <class K, int MB = NLINV_PMINB>
__global__ void __launch_bounds__(K::BS, MB) kf_coil_y(Ctx C0, PhaseBatch B) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  extern __shared__ float2 sm[];
  phase_coil_y<K>(C, sm, C.xn + (size_t)C.N * C.N, C.h);
}

// ROW_COIL: coil maps and rho c_j rows through the padded row FFT;
// ROW_COILONLY: the coil maps alone
template <class K, int MB = NLINV_PMINB>
__global__ void __launch_bounds__(K::BS, MB) kf_row_b(Ctx C0, PhaseBatch B, int mode) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  extern __shared__ float2 sm[];
  if (mode == ROW_COIL)
    phase_row_b<K>(C, sm, ROW_COIL, C.h, C.xn, nullptr, nullptr, C.v);
  else
    phase_row_b<K>(C, sm, ROW_COILONLY, C.h, nullptr, nullptr, nullptr, nullptr);
}

// COL_RHS: column pass of the residual against the frame's data;
// COL_TOEP: the PSF column pass of a CG iteration (both with the frame's PSF)
// (one kernel per mode, so each compiles for its own operands: the CG's PSF
// pass needs 233 registers at one CTA per SM, none spilled at 128; with
// K::OMINB two CTAs per SM where they fit, as for the row pass back)
template <class K, int MODE>
__global__ void __launch_bounds__(K::BS, MODE == COL_TOEP ? K::OMINB : NLINV_PMINB) kf_col_c(Ctx C0, PhaseBatch B,
                                                                                        int k) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  extern __shared__ float2 sm[];
  const FrameIO& io = B.io[f];
  phase_col_c<K>(C, sm, MODE, io.P, MODE == COL_RHS ? io.Y : nullptr, nullptr, C.v, k);
}

template <class K>
__global__ void __launch_bounds__(K::BS, K::OMINB) kf_row_d(Ctx C0, PhaseBatch B) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  extern __shared__ float2 sm[];
  phase_row_d<K>(C, sm, C.xn, C.v, C.s, C.kb);
}

// E_RHS: the Newton right-hand side r_0 (the last step regularised towards
// damping * x_last when `last` and the frame has one) and H r_0;
// E_CGR: w_k = A r_k, the partials of Re<r_k, w_k> and |r_k|^2, and H w_k
template <class K, int MODE, int MB = NLINV_PMINB>
__global__ void __launch_bounds__(K::BS, MB) kf_col_e(Ctx C0, PhaseBatch B, float alpha, int k,
                                                               int last, float damping) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  extern __shared__ float2 sm[];
  __shared__ float2 sred[32];
  if (MODE == E_RHS) {
    const float2* xl = last ? B.io[f].xlast : nullptr;
    phase_col_e<K, E_RHS>(C, sm, sred, alpha, 0, C.kb, C.s, nullptr, nullptr, C.rb[0], C.Hr, SLOT_RR0, xl,
                          xl ? damping : 1.f);
  } else {
    phase_col_e<K, E_CGR>(C, sm, sred, alpha, k, C.kb, C.s, nullptr, C.rb[k & 1], C.q, C.Hw, SLOT_PQ);
  }
}

// the row pass of r_k, with step k-1's update (phases_cgr.cuh)
template <class K, int MB = NLINV_PMINB>
__global__ void __launch_bounds__(K::BS, MB) kf_row_cgr(Ctx C0, PhaseBatch B, int k) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  extern __shared__ float2 sm[];
  phase_row_cgr<K>(C, sm, k);
}

// the CG's last step: x^_{n+1} = x^_n + x_K
template <class K>
__global__ void __launch_bounds__(K::BS, NLINV_PMINB) kf_cgr_final(Ctx C0, PhaseBatch B, int Kcg) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  phase_cgr_final<K>(C, Kcg);
}

// outputs: x^, rho, rho * sqrt(sum_j |c_j|^2)
__global__ void kf_final(Ctx C0, PhaseBatch B) {
  int f;
  const Ctx C = frame_entry(C0, B, f);
  const FrameIO& io = B.io[f];
  phase_final(C, io.xout, io.rho_out, io.img_out);
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

// ------------------------------------------ cluster-resident frame kernel
// One frame with one thread-block cluster per channel (cluster.cuh): per CG
// iteration the row and column passes of a channel meet at cluster barriers
// (their transposes are pushes into the owners' shared memory); only the
// channel sum and the two CG inner products use the grid barrier, twice per
// iteration.  Launched cooperatively (all clusters co-resident).  Errors never
// end a CTA early: every CTA runs every cluster barrier, so no CTA leaves
// while a peer may still store into its shared memory; an expired wait or a
// CG breakdown only latches the error word (the bounded grid barriers stop
// waiting once it is set).

// grid barrier that also orders this CTA's pushes for its cluster peers
__device__ __forceinline__ void gsync_cl(const Ctx& C, unsigned& epoch) {
  cl::arrive();
  grid_sync(C, epoch);
  cl::wait();
}

// CG step a = |r_k|^2 / Re<p_k, A p_k> from the partials, once per CTA
__device__ __forceinline__ Scal2 cta_step(const Ctx& C, int k) {
  __shared__ Scal2 s_a;
  if (threadIdx.x < 32) {
    const DF32 rrs = slot_sum(C, (k & 1) ? SLOT_RR1 : SLOT_RR0);
    const DF32 pqs = slot_sum(C, SLOT_PQ);
    if (threadIdx.x == 0) {
      const double rr = df_to_double(rrs);
      const double a64 = cg_step(rr, df_to_double(pqs));
      if (rr > 0.0 && a64 == 0.0) raise_err(C, DEV_ENUMERIC);
      const float hi = (float)a64;
      s_a = Scal2{hi, (float)(a64 - (double)hi)};
    }
  }
  __syncthreads();
  return s_a;
}

// The Newton right-hand side DF^H (Y - P F^(x^_n)) - alpha_n (x^_n - x_ref)
// and H r_0 (once per Newton step, against ten CG iterations): kept out of
// line so that its operand registers do not add to the CG loop's pressure.
template <class K>
__device__ __noinline__ void cl_rhs(const Ctx& C, const cl::Lay& L, float2* sm, float2* sred, const FrameIO& io,
                                    float al, unsigned& epoch) {
  const Scal2 zero{0.f, 0.f};
  float acc = 0.f, unused = 0.f;
  cl::coil_y<K>(C, L, sm, C.xn + C.N * C.N);
  cl::csync();
  cl::row_b<K>(C, L, sm, ROW_COIL);
  cl::csync();
  cl::col_c<K>(C, L, sm, COL_RHS, io.P, io.Y, zero, true);
  cl::csync();
  cl::row_d<K>(C, L, sm, nullptr, nullptr, zero, true, unused);
  cl::csync();
  cl::col_e<K, E_RHS>(C, L, sm, al, zero, true, nullptr, nullptr, nullptr, C.rb[0], C.xref, 1.f, acc);
  gsync_cl(C, epoch);
  cl::rho_rhs(C, al, C.xref, 1.f, acc);
  block_partial(C, acc, SLOT_RR0, sred);
  gsync_cl(C, epoch);
}

template <class K>
__global__ void __launch_bounds__(K::BS, 1) k_frame_cl(Ctx C0, FrameArgs F, cl::Lay L) {
  extern __shared__ float2 sm[];
  __shared__ float2 sred[32];
  const Ctx C = whole_grid(C0);
  const int NN = C.N * C.N;
  unsigned epoch = 0;
  cl::csync();   // every CTA of the cluster runs before the first push
  phase_init(C, F.io.xprev, F.damping);
  gsync_cl(C, epoch);
  for (int n = 0; n < F.M; ++n) {
    const float al = F.alpha[n];
    cl_rhs<K>(C, L, sm, sred, F.io, al, epoch);
    for (int k = 0; k < F.K; ++k) {
      const bool first = (k == 0), last = (k == F.K - 1);
      const float2* rk = C.rb[k & 1];
      float2* rk1 = C.rb[(k + 1) & 1];
      float2* pk = C.pb[k & 1];
      const float2* pm = C.pb[(k + 1) & 1];
      const Scal2 beta = cta_beta(C, k);
      float pq = 0.f;
      cl::row_cg<K>(C, L, sm, rk);
      cl::rho_p(C, rk, pm, pk, beta, first, al, pq);
      cl::csync();
      cl::col_c<K>(C, L, sm, COL_CG, F.io.P, nullptr, beta, first);
      cl::csync();
      cl::row_d<K>(C, L, sm, rk, pm, beta, first, pq);
      cl::csync();
      cl::col_e<K, E_CG>(C, L, sm, al, beta, first, rk, pm, pk, nullptr, nullptr, 0.f, pq);
      block_partial(C, pq, SLOT_PQ, sred);
      gsync_cl(C, epoch);
      const Scal2 a = cta_step(C, k);
      float rr = 0.f;
      cl::upd_coil<K>(C, L, sm, a, first, last, rk, rk1, pk, rr);
      cl::rho_upd(C, a, first, last, al, rk, rk1, pk, rr);
      if (!last) block_partial(C, rr, (k & 1) ? SLOT_RR0 : SLOT_RR1, sred);
      gsync_cl(C, epoch);
    }
  }
  cl::coil_y<K>(C, L, sm, C.xn + NN);
  cl::csync();
  cl::row_b<K>(C, L, sm, ROW_COILONLY);
  gsync_cl(C, epoch);
  phase_final(C, F.io.xout, F.io.rho_out, F.io.img_out);
  cl::csync();   // no CTA leaves while a peer could still address it
}

// Shared-memory layout of the cluster kernel for an N x N image, Gc coil
// grid and CS CTAs per cluster (cluster.cuh).
template <class K>
cl::Lay cluster_layout(int N, int Gc, int CS) {
  cl::Lay L;
  std::memset(&L, 0, sizeof(L));
  const int G = K::G;
  L.CS = CS;
  L.R = (N + CS - 1) / CS;
  L.C = (G + CS - 1) / CS;
  L.Cc = (Gc + CS - 1) / CS;
  int off = 0;
  auto take = [&](int n) {
    const int o = off;
    off += (n + 1) & ~1;   // 16-byte aligned buffers
    return o;
  };
  L.rb = take(L.R * K::RS);
  L.cb = take(N * L.C);
  L.xb = take(G * K::TW);
  L.hb = take(L.R * Gc);
  L.kb = take(N * L.Cc);
  L.cj = take(L.R * N);
  L.vo = take(N * L.C);
  L.smem_bytes = off * (int)sizeof(float2);
  return L;
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


#ifdef NLINV_TIMELINE
int read_timeline(unsigned long long* host, int n) {
  if (n > 160 * 1024) n = 160 * 1024;
  CK(cudaMemcpyFromSymbol(host, g_timeline, (size_t)n * sizeof(unsigned long long)));
  return NLINV_OK;
}
int read_stages(unsigned long long* ns, unsigned long long* cnt) {
  CK(cudaMemcpyFromSymbol(ns, nlinv::g_stage_ns, sizeof(unsigned long long) * 64));
  CK(cudaMemcpyFromSymbol(cnt, nlinv::g_stage_n, sizeof(unsigned long long) * 64));
  return NLINV_OK;
}
#endif


// Dynamic shared memory for the two-CTA phase kernels (kf_col_c of the CG,
// kf_row_d) in a one-frame launch: more than half of an SM's, so that one CTA
// sits on each SM.  A lone frame's 152 CTAs, launched early behind their
// predecessor, otherwise pair up on the SMs that free first (measured 2.97
// against 2.76 ms per frame); frames of a batch keep two per SM (C3 396 ->
// 432 frames/s).
constexpr int kOneCtaSmem = 116 * 1024;
template <class K>
constexpr int one_cta_smem() {
  return K::OMINB == 2 ? (K::SMEM > kOneCtaSmem ? K::SMEM : kOneCtaSmem) : K::SMEM;
}

template <class K>
int set_smem_attrs() {
  if (one_cta_smem<K>() > 48 * 1024) {
    CK(cudaFuncSetAttribute(kf_col_c<K, COL_TOEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, one_cta_smem<K>()));
    CK(cudaFuncSetAttribute(kf_row_d<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, one_cta_smem<K>()));
  }
  if (K::SMEM > 48 * 1024) {
    CK(cudaFuncSetAttribute(k_coil_y<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_row_b<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_row_deapod<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_col_c<K, COL_TOEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_col_c<K, COL_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_col_c<K, COL_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_row_d<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_col_e<K, E_DFH>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_col_e<K, E_NORMAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_coil_y<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_row_b<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_coil_y<K, K::OMINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_row_b<K, K::OMINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_cgr_final<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_col_c<K, COL_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_col_e<K, E_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_col_e<K, E_CGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_row_cgr<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_col_e<K, E_CGR, K::OMINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(kf_row_cgr<K, K::OMINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_frame<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
    CK(cudaFuncSetAttribute(k_batch<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM));
  }
  return NLINV_OK;
}

// launch configuration of the cluster kernel: CS CTAs per cluster, J clusters
cudaLaunchConfig_t cluster_config(const nlinv_plan_s* pl, int CS, int bs, int smem, cudaLaunchAttribute* at,
                                  cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(pl->J * CS);
  cfg.blockDim = dim3(bs);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cfg;
}

// The largest cluster size (CTAs per channel) whose layout fits the shared
// memory of one CTA and whose J clusters are co-resident, or none (cl_cs = 0);
// the plan's cluster_cs, when set, is the only size tried.
template <class K>
int pick_cluster(nlinv_plan_s* pl) {
  static const int cand[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2, 1};
  const int only = pl->prm.cluster_cs;
  int optin = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->dev));
  // one attribute value for every plan of this grid size: the largest
  // dynamic size any layout may take (each launch passes its own size)
  const int max_dyn = optin - 1024;
  CK(cudaFuncSetAttribute(k_frame_cl<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn));
  CK(cudaFuncSetAttribute(k_frame_cl<K>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  pl->cl_cs = 0;
  for (int CS : cand) {
    if (only > 0 && CS != only) continue;
    if ((long long)pl->J * CS > kMaxPart) continue;
    const cl::Lay L = cluster_layout<K>(pl->N, pl->Gc, CS);
    if (L.smem_bytes > max_dyn) continue;
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config(pl, CS, K::BS, L.smem_bytes, at, nullptr);
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (const void*)k_frame_cl<K>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (ncl >= pl->J) {
      pl->cl_cs = CS;
      pl->cl_lay = L;
      return NLINV_OK;
    }
  }
  return NLINV_OK;
}

// launch helpers for the one-launch-per-phase path
template <class K>
struct Launch {
  const nlinv_plan_s* pl;
  cudaStream_t st;
  int fixed = 0;   // if > 0: every launch uses this many CTAs (CG reductions need equal counts)
  bool pdl = false;   // launch with programmatic dependent launch (see phase_entry)
  int pick(int g) const { return fixed > 0 ? fixed : (pl->op_grid > 0 && g > pl->op_grid ? pl->op_grid : g); }
  template <class... KArgs, class... Args>
  int go(void (*kern)(KArgs...), int grid, int block, size_t smem, const char* what, Args... args) const {
    if (!pdl) {
      kern<<<grid, block, smem, st>>>(args...);
      CKL(what);
      return NLINV_OK;
    }
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, kern, args...));
    return NLINV_OK;
  }
  int coil_y(const float2* src, float2* hout) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.Gc + K::TW - 1) / K::TW), 1);
    return go(&k_coil_y<K>, pick(g), K::BS, (size_t)K::SMEM, "k_coil_y", C, src, hout);
  }
  int row_b(int mode, const float2* hin, const float2* rho, const float2* drho, const float2* img,
            float2* vout) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.N + K::TW - 1) / K::TW), 1);
    return go(&k_row_b<K>, pick(g), K::BS, (size_t)K::SMEM, "k_row_b", C, mode, hin, rho, drho, img, vout);
  }
  int row_deapod(const float* dap, float scale, float2* v) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.N + K::TW - 1) / K::TW), 1);
    return go(&k_row_deapod<K>, pick(g), K::BS, (size_t)K::SMEM, "k_row_deapod", C, dap, scale, v);
  }
  int col_c(int mode, const float* P, const float2* Yin, float2* zout, float2* vio, int k = 0) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.G + K::TW - 1) / K::TW), 1);
    const size_t sm = (size_t)K::SMEM;
    switch (mode) {
      case COL_TOEP: return go(&k_col_c<K, COL_TOEP>, pick(g), K::BS, sm, "k_col_c", C, P, Yin, zout, vio, k);
      case COL_FWD: return go(&k_col_c<K, COL_FWD>, pick(g), K::BS, sm, "k_col_c", C, P, Yin, zout, vio, k);
      case COL_INV: return go(&k_col_c<K, COL_INV>, pick(g), K::BS, sm, "k_col_c", C, P, Yin, zout, vio, k);
      default: return NLINV_EINVAL;
    }
  }
  int row_d(const float2* rho, const float2* win, float2* sout, float2* kbout) const {
    const Ctx& C = pl->C;
    const int g = plan_grid(C.J * ((C.N + K::TW - 1) / K::TW), 1);
    return go(&k_row_d<K>, pick(g), K::BS, (size_t)K::SMEM, "k_row_d", C, rho, win, sout, kbout);
  }
  int col_e(int mode, float alpha, int k, const float2* kbin, const float2* sin, const float2* p_old,
            float2* p_new, float2* out, float2* hout, int slot) const {
    const Ctx& C = pl->C;
    const int items = C.J * ((C.Gc + K::TW - 1) / K::TW);
    const int g = plan_grid(items, (C.N * C.N + K::BS - 1) / K::BS);
    const size_t sm = (size_t)K::SMEM;
    switch (mode) {
      case E_DFH:
        return go(&k_col_e<K, E_DFH>, pick(g), K::BS, sm, "k_col_e", C, alpha, k, kbin, sin, p_old, p_new, out, hout,
                  slot);
      case E_NORMAL:
        return go(&k_col_e<K, E_NORMAL>, pick(g), K::BS, sm, "k_col_e", C, alpha, k, kbin, sin, p_old, p_new, out,
                  hout, slot);
      default: return NLINV_EINVAL;
    }
  }
  // coil maps c_j = W^-1 c^_j of x^ into the plan's c buffer
  int coils(const float2* xhat) const {
    const Ctx& C = pl->C;
    int rc = coil_y(xhat + (size_t)C.N * C.N, C.h);
    if (rc) return rc;
    return row_b(ROW_COILONLY, C.h, nullptr, nullptr, nullptr, nullptr);
  }
};


// ------------------------------------------------- constant twiddle table
// c_tw lives in this unit's module: upload it once per device.
std::mutex g_tw_mu;
bool g_tw_ready[64] = {};

int ensure_constants() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tw_mu);
  if (dev < 0 || dev >= 64) return NLINV_EINVAL;
  if (g_tw_ready[dev]) return NLINV_OK;
  float2 h[TWL];
  int off = 0;
  for (int i = 0; i < kNumTwLens; ++i) {   // block L: exp(-2 pi i e / L), e < L
    const int L = kTwLens[i];
    for (int e = 0; e < L; ++e) {
      const double a = -2.0 * M_PI * (double)e / L;
      h[off + e] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    off += L;
  }
  CK(cudaMemcpyToSymbol(c_tw, h, sizeof(h)));
  g_tw_ready[dev] = true;
  return NLINV_OK;
}

// ------------------------------------------------------ the operations
template <class K>
struct Ops {
  static int prepare() {
    RC(ensure_constants());
    return set_smem_attrs<K>();
  }

  static int setup(nlinv_plan_s* pl) {
    RC(prepare());
    int nbk = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, k_frame<K>, K::BS, K::SMEM));
    int g = nbk * pl->nsm;
    if (g > kMaxPart) g = kMaxPart;
    pl->coop_grid = g;
    int nbb = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbb, k_batch<K>, K::BS, K::SMEM));
    pl->batch_occ = nbb;
    // one-phase launches: the co-resident CTAs of the phase kernels, but no
    // more than the largest phase has items (+ the elementwise share)
    int occ = 1 << 20;
    const void* kf[] = {(const void*)kf_coil_y<K>,          (const void*)kf_row_b<K>,
                        (const void*)kf_col_c<K, COL_TOEP>, (const void*)kf_col_c<K, COL_RHS>,
                        (const void*)kf_row_d<K>,           (const void*)kf_col_e<K, E_RHS>,
                        (const void*)kf_col_e<K, E_CGR>,    (const void*)kf_row_cgr<K>,
                        (const void*)kf_cgr_final<K>};
    for (const void* fn : kf) {
      int o = 0;
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, K::BS, K::SMEM));
      occ = o < occ ? o : occ;
    }
    const int most = pl->J * ((pl->G + K::TW - 1) / K::TW) + kElemCTAs;
    // a frame whose row passes alone have items for two rounds of two CTAs
    // per SM runs its phases like a batch: the two-CTA variants and twice
    // the CTAs per frame
    const int ritems = pl->J * ((pl->N + K::TW - 1) / K::TW);
    pl->dense = K::OMINB == 2 && ritems >= 4 * K::OMINB * pl->nsm;
    if (pl->dense) occ = K::OMINB;
    int pg = occ * pl->nsm;
    if (pg > most) pg = most;
    if (pg > kMaxPart) pg = kMaxPart;
    pl->phase_grid = pg;
    pl->op_minb = K::OMINB;
    // the CG's PSF column pass deposits and reads no partial sums, so it may
    // run its own CTA count: one CTA per item as far as the co-resident CTAs
    // allow (at C2, 270 items in one round at two CTAs per SM instead of two
    // rounds of 152)
    int oc = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, kf_col_c<K, COL_TOEP>, K::BS, K::SMEM));
    const int citems = pl->J * ((pl->G + K::TW - 1) / K::TW);
    int cg = oc * pl->nsm;
    if (cg > citems) cg = citems;
    if (cg < pg) cg = pg;
    pl->colc_grid = cg;
    if (pg <= 0) return NLINV_ECUDA;
    if (pl->prm.exec_mode == 3) {
      RC(pick_cluster<K>(pl));
      if (pl->cl_cs == 0) return NLINV_EUNSUPPORTED;
    }
    return (g > 0 && nbb > 0) ? NLINV_OK : NLINV_ECUDA;
  }

  static int coils(const nlinv_plan_s* pl, cudaStream_t st, const float2* x) {
    Launch<K> L{pl, st};
    return L.coils(x);
  }

  static int DF(const nlinv_plan_s* pl, cudaStream_t st, const float2* x, const float2* d, float2* z,
                bool coils_ready) {
    Launch<K> L{pl, st};
    const size_t NN = (size_t)pl->N * pl->N;
    if (!coils_ready) RC(L.coils(x));
    RC(L.coil_y(d + NN, pl->C.h));
    RC(L.row_b(ROW_LIN, pl->C.h, x, d, nullptr, pl->C.v));
    return L.col_c(COL_FWD, nullptr, nullptr, z, pl->C.v);
  }

  static int DFH(const nlinv_plan_s* pl, cudaStream_t st, const float2* x, const float2* z, float2* out,
                 bool coils_ready) {
    Launch<K> L{pl, st};
    if (!coils_ready) RC(L.coils(x));
    RC(L.col_c(COL_INV, nullptr, z, nullptr, pl->C.v));
    RC(L.row_d(x, pl->C.v, pl->C.s, pl->C.kb));
    return L.col_e(E_DFH, 0.f, 0, pl->C.kb, pl->C.s, nullptr, nullptr, out, nullptr, SLOT_PQ);
  }

  static int normal(const nlinv_plan_s* pl, cudaStream_t st, const float2* x, const float2* d, const float* P,
                    double alpha, float2* out, bool coils_ready) {
    Launch<K> L{pl, st};
    const size_t NN = (size_t)pl->N * pl->N;
    if (!coils_ready) RC(L.coils(x));
    RC(L.coil_y(d + NN, pl->C.h));
    RC(L.row_b(ROW_LIN, pl->C.h, x, d, nullptr, pl->C.v));
    RC(L.col_c(COL_TOEP, P, nullptr, nullptr, pl->C.v));
    RC(L.row_d(x, pl->C.v, pl->C.s, pl->C.kb));
    return L.col_e(E_NORMAL, (float)alpha, 0, pl->C.kb, pl->C.s, nullptr, (float2*)d, out, nullptr, SLOT_PQ);
  }

  static int grid_fwd(const nlinv_plan_s* pl, cudaStream_t st, float2* Y) {
    Launch<K> L{pl, st};
    RC(L.row_b(ROW_IMG, nullptr, nullptr, nullptr, pl->C.s, pl->C.v));
    return L.col_c(COL_FWD, nullptr, nullptr, Y, pl->C.v);
  }

  static int grid_kb(const nlinv_plan_s* pl, cudaStream_t st, const float2* Z, const float* dap, float scale,
                     float2* Y) {
    Launch<K> L{pl, st};
    RC(L.col_c(COL_INV, nullptr, Z, nullptr, pl->C.v));
    RC(L.row_deapod(dap, scale, pl->C.v));
    return L.col_c(COL_FWD, nullptr, nullptr, Y, pl->C.v);
  }

  static int frame(const nlinv_plan_s* pl, cudaStream_t st, const FrameArgs& F) {
    const int mode = pl->prm.exec_mode;
    Ctx C = pl->C;
    if (mode == 3 && pl->cl_cs > 0) {
      CK(cudaMemsetAsync(C.bar, 0, 2 * sizeof(unsigned), st));
      cudaLaunchAttribute at[2];
      cudaLaunchConfig_t cfg = cluster_config(pl, pl->cl_cs, K::BS, pl->cl_lay.smem_bytes, at, st);
      CK(cudaLaunchKernelEx(&cfg, k_frame_cl<K>, C, F, pl->cl_lay));
      return NLINV_OK;
    }
    if (mode == 2) {
      CK(cudaMemsetAsync(C.bar, 0, 2 * sizeof(unsigned), st));
      FrameArgs Fa = F;
      void* args[] = {(void*)&C, (void*)&Fa};
      CK(cudaLaunchCooperativeKernel((const void*)k_frame<K>, dim3(pl->coop_grid), dim3(K::BS), args,
                                     (size_t)K::SMEM, st));
      return NLINV_OK;
    }
    return phased_run(const_cast<nlinv_plan_s*>(pl), st, &F.io, 1, F.M, F.K, F.damping, F.alpha);
  }

  // nf frames of the plan as one launch per fused phase, each launch over
  // all frames (frame_entry); the frames' inputs and outputs are read from
  // the plan's device table io_dev.  Optionally with programmatic dependent
  // launches between the kernels.
  static int phased(const nlinv_plan_s* pl, cudaStream_t st, int nf, int M, int Kcg, float damping,
                    const float* alpha, bool pdl) {
    const Ctx& C = pl->C;
    Launch<K> L{pl, st, 0, pdl};
    // CTAs per frame: a batch spreads two waves of resident CTAs over its
    // frames (fewer, busier CTAs: each pays the step scalars and the launch
    // once for more items; C3 524 -> 565 frames/s against one frame's count)
    const int slots = 2 * K::OMINB * pl->nsm;
    auto per_frame = [&](int one) {
      if (nf == 1) return one;
      const int b = (slots + nf - 1) / nf;
      return b < one ? (b > 0 ? b : 1) : one;
    };
    const PhaseBatch B{pl->fstride, per_frame(pl->phase_grid), pl->io_dev};
    const PhaseBatch Be{pl->fstride, plan_grid((int)((C.nx + 255) / 256), 1), pl->io_dev};
    const PhaseBatch Bc{pl->fstride, per_frame(pl->colc_grid), pl->io_dev};
    const int gp = nf * B.nbf, ge = nf * Be.nbf, gc = nf * Bc.nbf;
    const size_t sm = (size_t)K::SMEM;
    const bool two = nf > 1 || pl->dense;   // the two-CTA variants
    const size_t sm2 = two ? sm : (size_t)one_cta_smem<K>();   // kf_row_d (and kf_col_c at 1 CTA per SM)
    const size_t smc = (!two && Bc.nbf <= pl->nsm) ? sm2 : sm;
    RC(L.go(&kf_init, ge, 256, 0, "kf_init", C, Be, damping));
    for (int n = 0; n < M; ++n) {
      const float al = alpha[n];
      if (two) {
        RC(L.go(&kf_coil_y<K, K::OMINB>, gp, K::BS, sm, "kf_coil_y", C, B));
        RC(L.go(&kf_row_b<K, K::OMINB>, gp, K::BS, sm, "kf_row_b", C, B, (int)ROW_COIL));
      } else {
        RC(L.go(&kf_coil_y<K>, gp, K::BS, sm, "kf_coil_y", C, B));
        RC(L.go(&kf_row_b<K>, gp, K::BS, sm, "kf_row_b", C, B, (int)ROW_COIL));
      }
      RC(L.go(&kf_col_c<K, COL_RHS>, gp, K::BS, sm, "kf_col_c", C, B, 0));
      RC(L.go(&kf_row_d<K>, gp, K::BS, sm2, "kf_row_d", C, B));
      RC(L.go(&kf_col_e<K, E_RHS>, gp, K::BS, sm, "kf_col_e", C, B, al, 0, n == M - 1 ? 1 : 0, damping));
      // CG with the operator applied to the residual: four phases per iteration
      for (int k = 0; k < Kcg; ++k) {
        if (two)
          RC(L.go(&kf_row_cgr<K, K::OMINB>, gp, K::BS, sm, "kf_row_cgr", C, B, k));
        else
          RC(L.go(&kf_row_cgr<K>, gp, K::BS, sm, "kf_row_cgr", C, B, k));
        RC(L.go(&kf_col_c<K, COL_TOEP>, gc, K::BS, smc, "kf_col_c", C, Bc, k));
        RC(L.go(&kf_row_d<K>, gp, K::BS, sm2, "kf_row_d", C, B));
        if (two)
          RC(L.go(&kf_col_e<K, E_CGR, K::OMINB>, gp, K::BS, sm, "kf_col_e", C, B, al, k, 0, damping));
        else
          RC(L.go(&kf_col_e<K, E_CGR>, gp, K::BS, sm, "kf_col_e", C, B, al, k, 0, damping));
      }
      if (Kcg > 0) RC(L.go(&kf_cgr_final<K>, gp, K::BS, 0, "kf_cgr_final", C, B, Kcg));   // no dynamic smem
    }
    RC(L.go(&kf_coil_y<K>, gp, K::BS, sm, "kf_coil_y", C, B));
    RC(L.go(&kf_row_b<K>, gp, K::BS, sm, "kf_row_b", C, B, (int)ROW_COILONLY));
    return L.go(&kf_final, ge, 256, 0, "kf_final", C, Be);
  }

  // Frames io[0..nf) of the plan on the per-phase path: their table is
  // written to the device (as a kernel argument, so the host array may be
  // reused at once), then the phase sequence runs -- launched one kernel at
  // a time (exec_mode 1) or replayed from a CUDA graph captured once per
  // frame count and alpha_0 (exec_mode 0 and 4).
  static int phased_run(nlinv_plan_s* pl, cudaStream_t st, const FrameIO* io, int nf, int M, int Kcg,
                        float damping, const float* alpha) {
    if (nf <= 0 || nf > kMaxBatch || nf > pl->max_batch) return NLINV_EINVAL;
    if (!pl->io_dev) CK(cudaMalloc(&pl->io_dev, kMaxBatch * sizeof(FrameIO)));
    IOTable T;
    std::memset(&T, 0, sizeof(T));
    for (int f = 0; f < nf; ++f) T.io[f] = io[f];
    k_set_io<<<1, kMaxBatch, 0, st>>>(T, nf, pl->io_dev);
    CKL("k_set_io");
    if (pl->prm.exec_mode == 1) return phased(pl, st, nf, M, Kcg, damping, alpha, false);
    nlinv_plan_s::PhaseGraph* g = nullptr;
    for (auto& e : pl->pgraphs)
      if (e.nf == nf) g = &e;
    if (!g) {
      pl->pgraphs.emplace_back();
      g = &pl->pgraphs.back();
      g->nf = nf;
    }
    if (!g->exec || g->alpha0 != pl->prm.alpha0) {
      if (g->exec) {
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
      }
      if (!pl->gcap) CK(cudaStreamCreateWithFlags(&pl->gcap, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(pl->gcap, cudaStreamCaptureModeThreadLocal));
      const int rc = phased(pl, pl->gcap, nf, M, Kcg, damping, alpha, true);
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(pl->gcap, &graph);
      if (rc != NLINV_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      CK(ec);
      const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
      cudaGraphDestroy(graph);
      CK(ei);
      g->alpha0 = pl->prm.alpha0;
    }
    CK(cudaGraphLaunch(g->exec, st));
    return NLINV_OK;
  }

  static int batch(const nlinv_plan_s* pl, cudaStream_t st, const BatchArgs& B, int grid) {
    const int mode = pl->prm.exec_mode;
    bool waits = false;
    for (int f = 0; f < B.nf; ++f) waits = waits || B.io[f].wait || B.io[f].done;
    if ((mode == 0 || mode == 1 || mode == 4) && !waits)
      return phased_run(const_cast<nlinv_plan_s*>(pl), st, B.io, B.nf, B.M, B.K, B.damping, B.alpha);
    Ctx C = pl->C;
    BatchArgs Ba = B;
    CK(cudaMemsetAsync(C.bar, 0, (size_t)B.nf * kBarStride * sizeof(unsigned), st));
    void* args[] = {(void*)&C, (void*)&Ba};
    CK(cudaLaunchCooperativeKernel((const void*)k_batch<K>, dim3(grid), dim3(K::BS), args, (size_t)K::SMEM, st));
    return NLINV_OK;
  }
};

template <class K>
const GridOps* make_ops() {
  static const GridOps ops = {K::G, K::NR, &Ops<K>::setup, &Ops<K>::prepare, &Ops<K>::coils, &Ops<K>::DF,
                              &Ops<K>::DFH, &Ops<K>::normal, &Ops<K>::grid_fwd, &Ops<K>::grid_kb, &Ops<K>::frame, &Ops<K>::batch
#ifdef NLINV_TIMELINE
                              , &read_timeline, &read_stages
#endif
  };
  return &ops;
}

}  // namespace
}  // namespace nlinv
