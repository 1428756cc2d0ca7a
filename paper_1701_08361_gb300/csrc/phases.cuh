// Device phases of the NLINV hot path (Schaetz et al. 2017, Sec. 2.2,
// Eqs. (2)-(5), Fig. 4) on one GB300.
//
// One application of the normal operator  DF^H P DF + alpha I  (Eq. (4)-(5)
// with the non-uniform pair replaced by the PSF multiplier P on the twofold
// grid) is five passes over per-channel data; each pass is one fused kernel
// phase and every pass keeps its 1-D FFTs in registers (see fft.cuh):
//
//   A  coil_y : W^-1 along y.  c^_j columns (G_c nonzero of G) -> N rows.
//   B  row_b  : W^-1 along x, then u_j = c_j drho + rho dc_j, then the
//               forward FFT of the zero-padded row (N nonzero of G).
//   C  col_c  : along y: FFT (N nonzero of G), x P / G^2, inverse FFT, keep
//               N rows -- the whole PSF convolution of a column in one go.
//   D  row_d  : inverse FFT along x, keep N: t_j.  s_j = conj(c_j) t_j is
//               stored for the channel sum; conj(rho) t_j is FFT'd along x and
//               cropped to the G_c coil band.
//   E  col_e  : FFT along y, crop to G_c, x D_W^-1: the W^-H part; plus the
//               channel sum  sum_j s_j  for the rho part; plus the Tikhonov
//               term and the CG inner product Re<p, q> (partials).
//
// A CG iteration runs B as row_cg (the row pass of the residual r_k, whose y
// pass H r_k the previous update produced; the direction p_k is formed
// elementwise by CTAs without a row item), C as col_cg (T(p_k) = T(r_k) +
// beta_k T(p_{k-1}) from the stored T(p_{k-1}), then the PSF column pass),
// D, E, and
//   F  upd    : x += a p, r_{k+1} = r_k - a q, |r_{k+1}|^2 (partials), and
//               H r_{k+1} for the next row pass.
// Data layouts (complex64 interleaved, row-major):
//   x^ vector   : rho [N][N] followed by c^ [J][Gc][Gc]        (n_x elements)
//   c  (coils)  : [J][N][N]      h  : [J][N][Gc]   (after the y pass of W^-1)
//   v  (rows)   : [J][N][G]      s  : [J][N][N]    kb : [J][N][Gc]
//   P           : [U][G][G] real  D_W^-1 : [Gc][Gc] real
// The FOV occupies rows/cols [0, N) of the G grid; the c^ grid holds
// frequency f at index f mod Gc and at index f mod G of the G grid.
//
// Buffers written by one phase and read by another are read with ld.global.cg
// (L2, not L1) because the persistent kernel runs every phase in one launch.
#pragma once
#include "fft.cuh"

// phases are inlined into the persistent kernel unless NLINV_NOINLINE_PHASES
// is defined (separate functions get their own register allocation but cost
// more than they save here)
#ifdef NLINV_NOINLINE_PHASES
#define NLINV_PHASE __noinline__
#else
#define NLINV_PHASE __forceinline__
#endif
// elementwise parts: elements per thread per round, and the fewest CTAs left
// over for them before a phase splits its CTAs between items and elements
#ifndef NLINV_EU
#define NLINV_EU 2
#endif
#ifndef NLINV_ELEM_CTAS
#define NLINV_ELEM_CTAS 32
#endif
// the CG column pass stages T(r_k), T(p_{k-1}) in shared memory; the PSF
// tile is read into registers (staging it too measured 1 % slower: the
// larger carve-out leaves less L1 for register spills)
#ifndef NLINV_STAGE_PSF
#define NLINV_STAGE_PSF 0
#endif
// pause between two polls of a barrier counter: fewer reads of the counter's
// line while CTAs arrive (32 ns measured 1.7 % faster per frame than none)
#ifndef NLINV_BAR_SLEEP_NS
#define NLINV_BAR_SLEEP_NS 32
#endif

namespace nlinv {

#ifdef NLINV_TIMELINE
// profiling builds: per (phase, stage) summed durations over all CTAs' items
__device__ unsigned long long g_stage_ns[8][8];
__device__ unsigned long long g_stage_n[8][8];
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#define STG_BEGIN() unsigned long long stg_t0 = gtimer()
#define STG(ph, st)                                                   \
  do {                                                                \
    if (threadIdx.x == 0) {                                           \
      const unsigned long long t1 = gtimer();                         \
      atomicAdd(&g_stage_ns[ph][st], t1 - stg_t0);                    \
      atomicAdd(&g_stage_n[ph][st], 1ull);                            \
      stg_t0 = t1;                                                    \
    }                                                                 \
  } while (0)
#else
#define STG_BEGIN()
#define STG(ph, st)
#endif

constexpr int kMaxPart = 4096;     // max CTAs that deposit a reduction partial
enum { SLOT_PQ = 0, SLOT_RR0 = 1, SLOT_RR1 = 2, NSLOT = 4 };
enum { DEV_ETIMEOUT = -4, DEV_ENUMERIC = -5 };

enum RowMode { ROW_COIL = 0, ROW_COILONLY = 1, ROW_LIN = 2, ROW_IMG = 3 };
enum ColMode { COL_TOEP = 0, COL_RHS = 1, COL_FWD = 2, COL_INV = 3, COL_CG = 4 };
enum EMode { E_CG = 0, E_RHS = 1, E_DFH = 2, E_NORMAL = 3, E_CGR = 4 };

struct Ctx {
  int N, G, Gc, J, nx, U;
  float inv_G, inv_G2;
  const float2* tw;     // [G] exp(-2 pi i e / G)
  const float* dinv;    // [Gc][Gc]
  const float* psf;     // [U][G][G]
  float2 *c, *h, *v, *s, *kb;
  float2 *xn, *xref, *xcg, *q;
  float2* rb[2];        // CG residual r_k lives in rb[k & 1]
  float2* pb[2];        // CG direction p_k lives in pb[k & 1]
  float2* Hr;           // y pass of W^-1 applied to r: [J][N][Gc]
  float2* vold;         // row pass of the previous CG direction p_{k-1}: [J][N][G]
  // the per-phase path's CG (operator applied to the residual): s_k = A p_k
  // in sb[k & 1], H w_k and H s_k ([J][N][Gc]), and (gamma, a) of the last
  // two steps in cgs[2 (k & 1)], cgs[2 (k & 1) + 1], gamma_0 in cgs[4], the
  // stop flag in cgs[5]
  float2* sb[2];
  float2 *Hw, *Hs;
  double* cgs;
  float2* part;         // [NSLOT][kMaxPart] per-CTA partials (float pairs hi, lo)
  int* err;             // latched device error
  unsigned* bar;        // barrier counter of the CTAs working on this frame
  long long spin_limit;
  int bid, nb;          // this CTA's index within the CTAs working on this frame, and their count
};

// One compiled grid: G = G1 x G2 (the two register DFT lengths), the image
// side NR (the field of view, rows/cols [0, NR) of the G grid; G = 2 NR unless
// a grid G = 2 gamma N of Eq. (8) is chosen), the tile width TW (columns of a
// column item, rows of a row item) and the CTAs per SM MINB the persistent
// kernels are compiled for.  A CTA of TW x max(G1, G2) threads with 10 or
// more warps is capped at 168 registers a thread and its register DFTs
// spill; at 8 warps (2 per scheduler) a thread may hold 255.  On the 320
// grid 12-wide tiles (256 threads) measured 3.44 ms per frame against 3.84
// ms for 16-wide tiles (320 threads); the batched and the 512 grid sizes
// measured faster with 16-wide tiles.
template <int G1_, int G2_, int NR_ = G1_ * G2_ / 2, int TW_ = 16,
          int MINB_ = ((TW_ * (G1_ > G2_ ? G1_ : G2_) + 31) / 32 * 32 <= 256 ? 2 : 1)>
struct Cfg {
  static constexpr int G1 = G1_, G2 = G2_;
  static constexpr int G = G1 * G2;
  static constexpr int MX = G1 > G2 ? G1 : G2;
  static constexpr int TW = TW_;            // columns per tile / rows per group
  static constexpr int BS = (TW * MX + 31) / 32 * 32;   // threads per CTA (whole warps)
  static constexpr int RS = G + MX;         // smem stride of one row (float2)
  static constexpr int NR = NR_;            // image rows N
  // FOV pruning: an index a + G2 b (a < G2, b unrolled) lies in [0, NR) for
  // every a when b < B2F, for some a when b < B2; likewise a + G1 b with B1F, B1
  static constexpr int B2F = NR / G2, B2 = (NR + G2 - 1) / G2;
  static constexpr int B1F = NR / G1, B1 = (NR + G1 - 1) / G1;
  static constexpr int SMEM_X = TW * RS * 8;  // exchange buffer bytes
  // CTAs per SM the persistent kernel is compiled for (caps registers)
  static constexpr int MINB = MINB_;
  // staged operands of one column item of the CG column pass: T(r_k) and
  // T(p_{k-1}) tiles [N][TW] (and the PSF tile [G][TW] if staged).  One staging buffer:
  // a second one (a full item ahead) measured slower, as the larger shared
  // memory carve-out shrinks the L1 cache that holds the register spills.
  static constexpr int CT = 2 * NR * TW * 8 + (NLINV_STAGE_PSF ? G * TW * 4 : 0);
  static constexpr int SMEM_LIM = MINB == 1 ? 227 * 1024 : 228 * 1024 / MINB - 1024;
  static constexpr int NBUF = 1;
  static constexpr int SMEM = SMEM_X + NBUF * CT;  // dynamic smem bytes
  static_assert(SMEM <= SMEM_LIM, "staging buffer does not fit");
  // CTAs per SM the single-call operator kernels (DF, DF^H, the normal
  // operator: many of them run side by side on several streams) are compiled
  // for: two where two blocks of at most 256 threads fit the shared memory
  static constexpr int OMINB = (BS <= 256 && 2 * (SMEM + 1024) <= 228 * 1024) ? 2 : 1;
  static_assert(TW % 4 == 0 && (G % 2) == 0, "16-byte staging chunks (even rows of float2)");
  static_assert(2 * NR <= G, "the field of view is at most half the grid");
  // the block reductions use full-warp shuffles over blockDim / 32 warps
  static_assert(BS % 32 == 0, "threads per CTA must be a whole number of warps");
};

// a + G2 b < NR (b compile-time after unrolling: only the one ragged b tests a)
template <class K> __device__ __forceinline__ bool in2(int b, int a) {
  return b < K::B2F || (b < K::B2 && a + K::G2 * b < K::NR);
}
// a + G1 b < NR
template <class K> __device__ __forceinline__ bool in1(int b, int a) {
  return b < K::B1F || (b < K::B1 && a + K::G1 * b < K::NR);
}

__device__ __forceinline__ float2 ldcg(const float2* p) { return __ldcg(p); }

// The thread index as a value the compiler must read anew in every phase:
// with all phases inlined into one persistent kernel, index arithmetic that
// is invariant over the CG loop would otherwise be hoisted out of it and
// held live (or spilled) across every phase.
__device__ __forceinline__ int phase_tid() {
  int t;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
  return t;
}

// A CG scalar (computed in FP64) as an unevaluated float pair hi + lo, so
// that y + s x keeps s to ~48 bits at the cost of two FP32 FMAs (FP64
// arithmetic runs at a small fraction of the FP32 rate on this part).
struct Scal2 {
  float hi, lo;
};
__device__ __forceinline__ float2 axpy2(float2 x, Scal2 s, float2 y) {
  return make_float2(fmaf(s.hi, x.x, fmaf(s.lo, x.x, y.x)), fmaf(s.hi, x.y, fmaf(s.lo, x.y, y.y)));
}

// index of grid position pos in the G_c coil band, -1 outside: the band
// holds the (Gc + 1) / 2 frequencies 0, 1, ... and the Gc / 2 frequencies
// -1, -2, ... (unshifted order; Gc odd or even)
__device__ __forceinline__ int coef_index(int pos, int G, int Gc) {
  if (pos < ((Gc + 1) >> 1)) return pos;
  if (pos >= G - (Gc >> 1)) return pos - G + Gc;
  return -1;
}

// -------------------------------------------------------- reductions
// Sums are carried as unevaluated float pairs hi + lo (~48 significant bits)
// with Knuth's two-sum, so the hot path needs no FP64 instructions (FP64 runs
// at a small fraction of the FP32 rate on this part).
struct DF32 {
  float hi, lo;
};
__device__ __forceinline__ DF32 df_add(DF32 a, DF32 b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  const float hi = s + e;
  return DF32{hi, e - (hi - s)};
}
__device__ __forceinline__ DF32 df_shfl_down(DF32 a, int o) {
  return DF32{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ DF32 df_warp_sum(DF32 a) {   // fixed tree, valid in lane 0
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_down(a, o));
  return a;
}

// Deterministic grid reduction, producer side: this CTA's threads' values
// (fixed warp trees) become part[slot][bid].  Consumers (a later phase,
// after a barrier or in a later kernel with the same CTA count) add the nb
// partials themselves with slot_sum().
__device__ __forceinline__ void block_partial(const Ctx& C, float v, int slot, float2* sred) {
  DF32 a = df_warp_sum(DF32{v, 0.f});
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sred[w] = make_float2(a.hi, a.lo);
  __syncthreads();
  if (threadIdx.x == 0) {
    DF32 t{0.f, 0.f};
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = df_add(t, DF32{sred[i].x, sred[i].y});
    C.part[slot * kMaxPart + C.bid] = make_float2(t.hi, t.lo);
  }
  __syncthreads();
}

// Consumer side: every warp adds the nb partials of `slot` in the same fixed
// order (one round trip to L2, no block barrier) and gets the same total.
__device__ __forceinline__ DF32 slot_sum(const Ctx& C, int slot) {
  const int l = threadIdx.x & 31;
  const float2* src = C.part + slot * kMaxPart;
  DF32 a{0.f, 0.f};
  for (int base = 0; base < C.nb; base += 32 * 8) {
    float2 v[8];   // all loads of a round issued before any add (one L2 round trip)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * 32 + l;
      v[u] = (i < C.nb) ? __ldcg(src + i) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) a = df_add(a, DF32{v[u].x, v[u].y});
  }
  a = df_warp_sum(a);
  return DF32{__shfl_sync(0xffffffffu, a.hi, 0), __shfl_sync(0xffffffffu, a.lo, 0)};
}

__device__ __forceinline__ double df_to_double(DF32 a) { return (double)a.hi + (double)a.lo; }

// FP64 scalar computed by lane 0 of each warp, handed to the warp as a
// float pair (FP64 instructions are slow on this part: one lane, not all)
__device__ __forceinline__ Scal2 warp_scalar(double v, bool lane0) {
  float hi = 0.f, lo = 0.f;
  if (lane0) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  }
  return Scal2{__shfl_sync(0xffffffffu, hi, 0), __shfl_sync(0xffffffffu, lo, 0)};
}

// beta_k = |r_k|^2 / |r_{k-1}|^2 (0 for k == 0 or a zero old residual);
// warp 0 reads the partials, the other warps get the value through shared
// memory (one reader per CTA keeps the partials' cache lines cool)
__device__ __forceinline__ Scal2 cg_beta(const Ctx& C, int k);
__device__ __forceinline__ Scal2 cta_beta(const Ctx& C, int k) {
  __shared__ Scal2 s_beta;
  if (k == 0) return Scal2{0.f, 0.f};
  if (threadIdx.x < 32) {
    const Scal2 b = cg_beta(C, k);
    if (threadIdx.x == 0) s_beta = b;
  }
  __syncthreads();
  return s_beta;
}
__device__ __forceinline__ Scal2 cg_beta(const Ctx& C, int k) {
  if (k == 0) return Scal2{0.f, 0.f};
  const DF32 rk = slot_sum(C, (k & 1) ? SLOT_RR1 : SLOT_RR0);
  const DF32 rm = slot_sum(C, (k & 1) ? SLOT_RR0 : SLOT_RR1);
  const bool l0 = (threadIdx.x & 31) == 0;
  double b = 0.0;
  if (l0) {
    const double d = df_to_double(rm);
    b = d > 0.0 ? df_to_double(rk) / d : 0.0;
  }
  return warp_scalar(b, l0);
}

__device__ __forceinline__ void raise_err(const Ctx& C, int code) { atomicCAS(C.err, 0, code); }

// ------------------------------------------------ A: W^-1 along y (coil)
// H(src): D_W^-1, then the inverse DFT along y of each c^ column (G_c
// nonzero of G), keeping rows y < N, scaled by 1/G.  src: [J][Gc][Gc].
template <class K>
__device__ NLINV_PHASE void phase_coil_y(const Ctx& C, float2* sm, const float2* src, float2* hout) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW;
  const int N = C.N, Gc = C.Gc, J = C.J;
  const int t = phase_tid();
  const int tiles = (Gc + TW - 1) / TW;
  const int items = J * tiles;
  for (int it = C.bid; it < items; it += C.nb) {
    const int j = it / tiles;
    const int fx = (it - j * tiles) * TW + (t % TW);
    const bool colok = fx < Gc;
    {  // stage 1: thread (n1, c), inverse DFT over n2
      const int n1 = t / TW;
      if (n1 < G1) {
        float2 a[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          const int iy = coef_index(n1 + G1 * n2, G, Gc);
          float2 val = czero();
          if (colok && iy >= 0)
            val = cscale(ldcg(src + ((size_t)j * Gc + iy) * Gc + fx), __ldg(C.dinv + iy * Gc + fx));
          a[n2] = val;
        }
        dft<G2, true>(a);
#pragma unroll
        for (int k2 = 0; k2 < G2; ++k2) {
          float2 x = a[k2];
          if (k2) x = cmul(x, twg<true>(C.tw, n1 * k2));
          sm[(k2 * G1 + n1) * TW + (t % TW)] = x;
        }
      }
    }
    __syncthreads();
    {  // stage 2: thread (k2, c), inverse DFT over n1, keep y < N
      const int k2 = t / TW, cc = t % TW;
      if (k2 < G2 && colok) {
        float2 b[G1];
#pragma unroll
        for (int n1 = 0; n1 < G1; ++n1) b[n1] = sm[(k2 * G1 + n1) * TW + cc];
        dft<G1, true>(b);
#pragma unroll
        for (int k1 = 0; k1 < K::B2; ++k1) {
          const int y = k2 + G2 * k1;
          if (in2<K>(k1, k2)) hout[((size_t)j * N + y) * Gc + fx] = cscale(b[k1], C.inv_G);
        }
      }
    }
    __syncthreads();
  }
}

// CG step length a = |r|^2 / Re<p, A p> (0 when |r|^2 = 0 or on breakdown)
__device__ __forceinline__ double cg_step(double rr, double pq) {
  return (rr > 0.0 && pq > 0.0 && isfinite(pq)) ? rr / pq : 0.0;
}

// Work split of the phases that have a few items and an elementwise part:
// when at least kElemCTAs CTAs would be left over, CTAs [0, items) take one
// item each and the others the elementwise part, so the two run side by
// side; otherwise every CTA takes both in turn.
constexpr int kElemCTAs = NLINV_ELEM_CTAS;
struct Roles {
  bool items, elems;    // what this CTA does
  int istride;          // item stride
  int ebid, enb;        // this CTA's index / the CTA count of the elementwise part
};
__device__ __forceinline__ Roles roles(const Ctx& C, int items) {
  if (items > 0 && items + kElemCTAs <= C.nb)
    return C.bid < items ? Roles{true, false, items, 0, 1} : Roles{false, true, items, C.bid - items, C.nb - items};
  return Roles{true, true, C.nb, C.bid, C.nb};
}

// ------------------------------------- B: W^-1 along x, product, row FFT
// mode ROW_COIL    : c = W^-1 c^ stored, u = rho c
//      ROW_COILONLY: c stored, nothing else
//      ROW_LIN     : u = c drho + rho dc
//      ROW_IMG     : u = img (no coil part)
template <class K>
__device__ NLINV_PHASE void phase_row_b(const Ctx& C, float2* sm, int mode, const float2* hin,
                            const float2* rho, const float2* drho, const float2* img,
                            float2* vout) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, RS = K::RS;
  const int N = C.N, Gc = C.Gc, J = C.J;
  const int t = phase_tid();
  const int groups = (N + TW - 1) / TW;
  const int items = J * groups;
  for (int it = C.bid; it < items; it += C.nb) {
    const int j = it / groups;
    const int y0 = (it - j * groups) * TW;
    if (mode != ROW_IMG) {  // stage 1: thread (row, n1): inverse DFT over n2
      const int rr = t / G1, n1 = t % G1, y = y0 + rr;
      if (rr < TW && y < N) {
        float2 a[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          const int ix = coef_index(n1 + G1 * n2, G, Gc);
          a[n2] = (ix >= 0) ? ldcg(hin + ((size_t)j * N + y) * Gc + ix) : czero();
        }
        dft<G2, true>(a);
#pragma unroll
        for (int k2 = 0; k2 < G2; ++k2) {
          float2 x = a[k2];
          if (k2) x = cmul(x, twg<true>(C.tw, n1 * k2));
          sm[rr * RS + k2 * (G1 + 1) + n1] = x;
        }
      }
      __syncthreads();
    }
    // stage 2: thread (row, k2): inverse DFT over n1 -> x = k2 + G2 k1,
    // product, forward DFT over k1 (x = k2 + G2 k1 is the input index)
    const int rr = t / G2, k2 = t % G2, y = y0 + rr;
    const bool ok = rr < TW && y < N;
    float2 u[G1];
    if (ok) {
      float2 b[G1];
      if (mode != ROW_IMG) {
#pragma unroll
        for (int n1 = 0; n1 < G1; ++n1) b[n1] = sm[rr * RS + k2 * (G1 + 1) + n1];
        dft<G1, true>(b);
      }
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1) {
        u[k1] = czero();
        if (in2<K>(k1, k2)) {
          const int x = k2 + G2 * k1;
          const size_t ic = ((size_t)j * N + y) * N + x;
          const int ir = y * N + x;
          if (mode == ROW_COIL) {
            C.c[ic] = b[k1];
            u[k1] = cmul(ldcg(rho + ir), b[k1]);
          } else if (mode == ROW_COILONLY) {
            C.c[ic] = b[k1];
          } else if (mode == ROW_LIN) {
            u[k1] = cadd(cmul(ldcg(C.c + ic), ldcg(drho + ir)), cmul(ldcg(rho + ir), b[k1]));
          } else {
            u[k1] = ldcg(img + ic);
          }
        }
      }
      if (mode != ROW_COILONLY) {
        dft<G1, false>(u);
#pragma unroll
        for (int kb = 1; kb < G1; ++kb) u[kb] = cmul(u[kb], twg<false>(C.tw, k2 * kb));
      }
    }
    if (mode == ROW_COILONLY) {
      __syncthreads();
      continue;
    }
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int kb = 0; kb < G1; ++kb) sm[rr * RS + kb * (G2 + 1) + k2] = u[kb];
    }
    __syncthreads();
    {  // stage 3: thread (row, kb): forward DFT over k2 -> kb + G1 ka
      const int r3 = t / G1, kb = t % G1, y3 = y0 + r3;
      if (r3 < TW && y3 < N) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = sm[r3 * RS + kb * (G2 + 1) + a2];
        dft<G2, false>(d);
        float2* dst = vout + ((size_t)j * N + y3) * G;
#pragma unroll
        for (int ka = 0; ka < G2; ++ka) dst[kb + G1 * ka] = d[ka];
      }
    }
    __syncthreads();
  }
}

// ------------------------ row pass of the convolution gridding (Sec. 3.1)
// The spread grid after the column pass COL_INV holds, per row y < N, the
// inverse transform along y; here: inverse DFT along x (keep x < N), times
// scale * dap[x] * dap[y] (the deapodisation), forward DFT of the zero-padded
// row, all G outputs back into the same row of v.
template <class K>
__device__ NLINV_PHASE void phase_row_deapod(const Ctx& C, float2* sm, const float* dap, float scale, float2* v) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, RS = K::RS;
  const int N = C.N, J = C.J;
  const int t = phase_tid();
  const int groups = (N + TW - 1) / TW;
  const int items = J * groups;
  for (int it = C.bid; it < items; it += C.nb) {
    const int j = it / groups;
    const int y0 = (it - j * groups) * TW;
    {  // stage 1: thread (row, n1): inverse DFT over n2 of the whole row
      const int r1 = t / G1, n1 = t % G1, y1 = y0 + r1;
      if (r1 < TW && y1 < N) {
        float2 a[G2];
        const float2* src = v + ((size_t)j * N + y1) * G;
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) a[n2] = ldcg(src + n1 + G1 * n2);
        dft<G2, true>(a);
#pragma unroll
        for (int q2 = 0; q2 < G2; ++q2) {
          float2 x = a[q2];
          if (q2) x = cmul(x, twg<true>(C.tw, n1 * q2));
          sm[r1 * RS + q2 * (G1 + 1) + n1] = x;
        }
      }
    }
    __syncthreads();
    // stage 2: thread (row, k2): inverse DFT over n1 -> x = k2 + G2 k1 (< N),
    // deapodisation, forward DFT over k1 of the padded row
    const int rr = t / G2, k2 = t % G2, y = y0 + rr;
    const bool ok = rr < TW && y < N;
    float2 u[G1];
    if (ok) {
      float2 b[G1];
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = sm[rr * RS + k2 * (G1 + 1) + q1];
      dft<G1, true>(b);
      const float wy = scale * __ldg(dap + y);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1)
        u[k1] = in2<K>(k1, k2) ? cscale(b[k1], wy * __ldg(dap + k2 + G2 * k1)) : czero();
      dft<G1, false>(u);
#pragma unroll
      for (int kb = 1; kb < G1; ++kb) u[kb] = cmul(u[kb], twg<false>(C.tw, k2 * kb));
    }
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int kb = 0; kb < G1; ++kb) sm[rr * RS + kb * (G2 + 1) + k2] = u[kb];
    }
    __syncthreads();
    {  // stage 3: thread (row, kb): forward DFT over k2 -> kb + G1 ka
      const int r3 = t / G1, kb = t % G1, y3 = y0 + r3;
      if (r3 < TW && y3 < N) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = sm[r3 * RS + kb * (G2 + 1) + a2];
        dft<G2, false>(d);
        float2* dst = v + ((size_t)j * N + y3) * G;
#pragma unroll
        for (int ka = 0; ka < G2; ++ka) dst[kb + G1 * ka] = d[ka];
      }
    }
    __syncthreads();
  }
}

// --------------------------- B in a CG iteration: the row pass of r_k
// The row pass T (x pass of W^-1 on the y-transformed coil part, the
// product u = c d_rho + rho W^-1 d_c, forward row FFT) is linear, so
// T(p_k) = T(r_k) + beta_k T(p_{k-1}): the items transform r_k alone (its
// y pass H r_k comes exactly from the update phase) and the column phase
// adds beta_k T(p_{k-1}), an addition without cancellation (p_{k-1} is
// conjugate to r_k).  The items thus need no CG scalar.  The CTAs left over
// form p_k = r_k + beta_k p_{k-1} elementwise for the later phases.
template <class K>
__device__ NLINV_PHASE void phase_row_cg(const Ctx& C, float2* sm, float2* sred, int k, const float2* p_old,
                             float2* p_new, float2* vout) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, RS = K::RS;
  constexpr int EU = NLINV_EU;   // elements per thread per round of the elementwise part
  const int N = C.N, Gc = C.Gc, J = C.J;
  const int t = phase_tid();
  const float2* rk = C.rb[k & 1];
  STG_BEGIN();
  const int groups = (N + TW - 1) / TW;
  const int items = J * groups;
  const Roles R = roles(C, items);
  if (R.items) for (int it = C.bid; it < items; it += R.istride) {
    const int j = it / groups;
    const int y0 = (it - j * groups) * TW;
    // stage-2 operands (r_rho, c_j, rho rows) are requested with stage 1's
    const int rr = t / G2, k2 = t % G2, y = y0 + rr;
    const bool ok = rr < TW && y < N;
    float2 rv[K::B2], cv[K::B2], rh[K::B2];
#pragma unroll
    for (int k1 = 0; k1 < K::B2; ++k1) {
      rv[k1] = cv[k1] = rh[k1] = czero();
      if (ok && in2<K>(k1, k2)) {
        const int ir = y * N + k2 + G2 * k1;
        rv[k1] = ldcg(rk + ir);
        cv[k1] = ldcg(C.c + (size_t)j * N * N + ir);
        rh[k1] = ldcg(C.xn + ir);
      }
    }
    {  // stage 1: thread (row, n1): inverse DFT over n2 of the band of H r
      const int r1 = t / G1, n1 = t % G1, y1 = y0 + r1;
      if (r1 < TW && y1 < N) {
        float2 av[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          const int ix = coef_index(n1 + G1 * n2, G, Gc);
          av[n2] = ix >= 0 ? ldcg(C.Hr + ((size_t)j * N + y1) * Gc + ix) : czero();
        }
        dft<G2, true>(av);
#pragma unroll
        for (int q2 = 0; q2 < G2; ++q2) {
          float2 x = av[q2];
          if (q2) x = cmul(x, twg<true>(C.tw, n1 * q2));
          sm[r1 * RS + q2 * (G1 + 1) + n1] = x;
        }
      }
    }
    __syncthreads();
    STG(0, 1);
    // stage 2: thread (row, k2): inverse DFT over n1 -> dc at x = k2 + G2 k1;
    // u = c r_rho + rho dc; forward DFT over k1
    float2 u[G1];
    if (ok) {
      float2 b[G1];
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = sm[rr * RS + k2 * (G1 + 1) + q1];
      dft<G1, true>(b);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1)
        u[k1] = (k1 < K::B2 && in2<K>(k1, k2))
                    ? cadd(cmul(cv[k1 < K::B2 ? k1 : 0], rv[k1 < K::B2 ? k1 : 0]), cmul(rh[k1 < K::B2 ? k1 : 0], b[k1]))
                    : czero();
      dft<G1, false>(u);
#pragma unroll
      for (int kb = 1; kb < G1; ++kb) u[kb] = cmul(u[kb], twg<false>(C.tw, k2 * kb));
    }
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int kb = 0; kb < G1; ++kb) sm[rr * RS + kb * (G2 + 1) + k2] = u[kb];
    }
    __syncthreads();
    STG(0, 2);
    {  // stage 3: thread (row, kb): forward DFT over k2 -> kb + G1 ka
      const int r3 = t / G1, kb = t % G1, y3 = y0 + r3;
      if (r3 < TW && y3 < N) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = sm[r3 * RS + kb * (G2 + 1) + a2];
        dft<G2, false>(d);
        float2* dst = vout + ((size_t)j * N + y3) * G;
#pragma unroll
        for (int ka = 0; ka < G2; ++ka) dst[kb + G1 * ka] = d[ka];
      }
    }
    __syncthreads();
    STG(0, 3);
  }
  // p_k = r_k + beta_k p_{k-1} (p_0 = r_0) over the whole vector
  if (R.elems) {
    Scal2 beta{0.f, 0.f};
    bool need_beta = k > 0;
    const int stride = R.enb * blockDim.x;
    for (int base = R.ebid * blockDim.x; base < C.nx; base += EU * stride) {   // CTA-uniform
      float2 rv[EU], pv[EU];
#pragma unroll
      for (int u = 0; u < EU; ++u) {
        const int e = base + t + u * stride;
        rv[u] = pv[u] = czero();
        if (e < C.nx) {
          rv[u] = ldcg(rk + e);
          if (k > 0) pv[u] = ldcg(p_old + e);
        }
      }
      if (need_beta) {
        beta = cta_beta(C, k);
        need_beta = false;
      }
#pragma unroll
      for (int u = 0; u < EU; ++u) {
        const int e = base + t + u * stride;
        if (e < C.nx) p_new[e] = (k > 0) ? axpy2(pv[u], beta, rv[u]) : rv[u];
      }
    }
  }
}

// ------------------------------------------------- asynchronous staging
// global -> shared copies in 16-byte chunks through L2 only (cp.async.cg),
// grouped per column item so that later items' copies overlap earlier work
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// ------------------------------ C in a CG iteration: staged column pass
// Per (channel, column tile): T(p_k) = T(r_k) + beta_k T(p_{k-1}) (kept in
// vold for the next iteration), FFT_y, x P / G^2, iFFT_y, keep N rows (in
// place in v).  An item's operands are staged into shared memory with
// asynchronous copies (the first item's at the start of the phase, while
// beta's partials are read; the next item's as soon as the buffer is free,
// overlapping the last transform stage).
template <class K>
__device__ NLINV_PHASE void phase_col_cg(const Ctx& C, float2* sm, const float* P, float2* vio, int k) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, NR = K::NR, BS = K::BS, NBUF = K::NBUF;
  constexpr int tiles = (G + TW - 1) / TW;
  constexpr int CTF = K::CT / 8;   // float2 per staging buffer
  const int J = C.J;
  const int t = phase_tid();
  const int items = J * tiles;
  float2* const stg = sm + K::SMEM_X / 8;
  STG_BEGIN();
  // copies of item number n of this CTA into buffer n % NBUF (an empty group
  // when there is no such item, so the group count stays uniform)
  auto stage = [&](int n) {
    const int it = C.bid + n * C.nb;
    if (it < items) {
      const int j = it / tiles, x0 = (it - j * tiles) * TW;
      const int wv = G - x0 < TW ? G - x0 : TW;   // valid columns, a multiple of 4
      float2* sv = stg + (n % NBUF) * CTF;
      float2* so = sv + NR * TW;
      float* sp = (float*)(so + NR * TW);
      constexpr int CPR = TW / 2;   // chunks per row of a complex tile
      for (int i = t; i < NR * CPR; i += BS) {
        const int r = i / CPR, c = (i % CPR) * 2;
        if (c < wv) {
          const size_t g = ((size_t)j * NR + r) * G + x0 + c;
          cp_async16(sv + r * TW + c, vio + g);
          if (k > 0) cp_async16(so + r * TW + c, C.vold + g);
        }
      }
      if (NLINV_STAGE_PSF) {
        constexpr int CPP = TW / 4;   // chunks per row of the PSF tile
        for (int i = t; i < G * CPP; i += BS) {
          const int r = i / CPP, c = (i % CPP) * 4;
          if (c < wv) cp_async16(sp + r * TW + c, P + (size_t)r * G + x0 + c);
        }
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int n = 0; n < NBUF; ++n) stage(n);
  const Scal2 beta = (k > 0 && C.bid < items) ? cta_beta(C, k) : Scal2{0.f, 0.f};   // CTA-uniform
  STG(1, 0);
  for (int n = 0; C.bid + n * C.nb < items; ++n) {
    const int it = C.bid + n * C.nb;
    const int j = it / tiles, x0 = (it - j * tiles) * TW;
    const float2* sv = stg + (n % NBUF) * CTF;
    const float2* so = sv + NR * TW;
    const float* sp = (const float*)(so + NR * TW);
    const int k2 = t / TW, cc = t % TW;
    const bool ok = k2 < G2 && x0 + cc < G;
    float pv[G1];   // the PSF of this thread's stage-2 points, when not staged
    if (!NLINV_STAGE_PSF) {
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1) pv[k1] = ok ? __ldg(P + (size_t)(k2 + G2 * k1) * G + x0 + cc) : 0.f;
    }
    cp_async_wait<NBUF - 1>();
    __syncthreads();
    STG(1, 1);
    {  // stage 1: thread (n1, c): T(p_k) of the column (rows y = n1 + G1 n2 < N), forward DFT over n2
      const int n1 = t / TW, c = t % TW;
      if (n1 < G1 && x0 + c < G) {
        float2 a[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          a[n2] = czero();
          if (in1<K>(n2, n1)) {
            const int y = n1 + G1 * n2;
            a[n2] = sv[y * TW + c];
            if (k > 0) a[n2] = axpy2(so[y * TW + c], beta, a[n2]);
            C.vold[((size_t)j * NR + y) * G + x0 + c] = a[n2];
          }
        }
        dft<G2, false>(a);
#pragma unroll
        for (int q2 = 0; q2 < G2; ++q2) {
          float2 v = a[q2];
          if (q2) v = cmul(v, twg<false>(C.tw, n1 * q2));
          sm[(q2 * G1 + n1) * TW + c] = v;
        }
      }
    }
    __syncthreads();
    // stage 2: thread (k2, c): forward DFT over n1 -> k = k2 + G2 k1, x P / G^2,
    // inverse DFT over k1
    float2 b[G1];
    if (ok) {
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = sm[(k2 * G1 + q1) * TW + cc];
      dft<G1, false>(b);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1)
        b[k1] = cscale(b[k1], (NLINV_STAGE_PSF ? sp[(k2 + G2 * k1) * TW + cc] : pv[k1]) * C.inv_G2);
      dft<G1, true>(b);
#pragma unroll
      for (int m1 = 1; m1 < G1; ++m1) b[m1] = cmul(b[m1], twg<true>(C.tw, k2 * m1));
    }
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int m1 = 0; m1 < G1; ++m1) sm[(m1 * G2 + k2) * TW + cc] = b[m1];
    }
    __syncthreads();
    STG(1, 2);
    stage(n + NBUF);   // this item's staging buffer is free again
    {  // stage 3: thread (m1, c): inverse DFT over k2 -> y = m1 + G1 m2, keep y < N
      const int m1 = t / TW, c = t % TW;
      if (m1 < G1 && x0 + c < G) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = sm[(m1 * G2 + a2) * TW + c];
        dft<G2, true>(d);
#pragma unroll
        for (int m2 = 0; m2 < K::B1; ++m2)
          if (in1<K>(m2, m1)) vio[((size_t)j * NR + m1 + G1 * m2) * G + x0 + c] = d[m2];
      }
    }
    __syncthreads();
    STG(1, 3);
  }
  cp_async_wait<0>();
}

// ------------------------------------------ C: column pass (PSF convolution)
// COL_CG  : v = T(r_k) + beta_k T(p_{k-1}) = T(p_k), kept as the next
//           T(p_{k-1}), then as COL_TOEP (T: the row pass of the CG phase)
// COL_TOEP: FFT_y, x P / G^2, iFFT_y, keep N rows (in place in v)
// COL_RHS : FFT_y, z = (Y - P X / G) / G, iFFT_y, keep N rows
// COL_FWD : FFT_y, zout = X / G (full G rows), stop
// COL_INV : X = Yin / G (full G rows given), iFFT_y, keep N rows
template <class K>
__device__ NLINV_PHASE void phase_col_c(const Ctx& C, float2* sm, int mode, const float* P,
                            const float2* Yin, float2* zout, float2* vio, int k = 0) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW;
  const int N = C.N, J = C.J;
  const int t = phase_tid();
  constexpr int tiles = (G + TW - 1) / TW;
  const int items = J * tiles;
  STG_BEGIN();
  const bool cg = (mode == COL_CG);
  if (cg) mode = COL_TOEP;
  bool need_beta = cg && k > 0;
  Scal2 beta{0.f, 0.f};
  for (int it = C.bid; it < items; it += C.nb) {
    const int j = it / tiles;
    const int x = (it - j * tiles) * TW + (t % TW);
    const bool colok = x < G;
    const int k2 = t / TW, cc = t % TW;
    const bool ok = k2 < G2 && colok;
    // the PSF (and data) of this thread's stage-2 points are requested first
    float pv[G1];
    float2 yv[G1];
#pragma unroll
    for (int k1 = 0; k1 < G1; ++k1) {
      pv[k1] = 0.f;
      yv[k1] = czero();
      const size_t kk = (size_t)(k2 + G2 * k1) * G + x;
      if (ok && (mode == COL_TOEP || mode == COL_RHS)) pv[k1] = __ldg(P + kk);
      if (ok && mode == COL_RHS) yv[k1] = ldcg(Yin + (size_t)j * G * G + kk);
    }
    if (mode != COL_INV) {  // stage 1: thread (n1, c): forward DFT over n2 (y = n1 + G1 n2 < N)
      const int n1 = t / TW;
      const bool ld = n1 < G1 && colok;
      float2 a[G2], ao[K::B1];
#pragma unroll
      for (int n2 = 0; n2 < G2; ++n2) {
        const bool in = ld && in1<K>(n2, n1);
        a[n2] = in ? ldcg(vio + ((size_t)j * N + n1 + G1 * n2) * G + x) : czero();
        if (n2 < K::B1) ao[n2 < K::B1 ? n2 : 0] = (in && cg && k > 0) ? ldcg(C.vold + ((size_t)j * N + n1 + G1 * n2) * G + x) : czero();
      }
      if (need_beta) {   // CTA-uniform: first item of this CTA
        beta = cta_beta(C, k);
        need_beta = false;
      }
      if (ld && cg) {
#pragma unroll
        for (int n2 = 0; n2 < K::B1; ++n2) {
          if (!in1<K>(n2, n1)) continue;
          if (k > 0) a[n2] = axpy2(ao[n2], beta, a[n2]);
          C.vold[((size_t)j * N + n1 + G1 * n2) * G + x] = a[n2];
        }
      }
      if (ld) {
        dft<G2, false>(a);
#pragma unroll
        for (int q2 = 0; q2 < G2; ++q2) {
          float2 v = a[q2];
          if (q2) v = cmul(v, twg<false>(C.tw, n1 * q2));
          sm[(q2 * G1 + n1) * TW + (t % TW)] = v;
        }
      }
      __syncthreads();
    }
    STG(1, 1);
    // stage 2: thread (k2, c): forward DFT over n1 -> k = k2 + G2 k1; the
    // pointwise step; inverse DFT over k1 (k = k2 + G2 k1 is the input index)
    float2 b[G1];
    if (ok) {
      if (mode == COL_INV) {
#pragma unroll
        for (int k1 = 0; k1 < G1; ++k1)
          b[k1] = cscale(ldcg(Yin + ((size_t)j * G + k2 + G2 * k1) * G + x), C.inv_G);
      } else {
#pragma unroll
        for (int n1 = 0; n1 < G1; ++n1) b[n1] = sm[(k2 * G1 + n1) * TW + cc];
        dft<G1, false>(b);
#pragma unroll
        for (int k1 = 0; k1 < G1; ++k1) {
          const size_t kk = (size_t)(k2 + G2 * k1) * G + x;
          if (mode == COL_TOEP) {
            b[k1] = cscale(b[k1], pv[k1] * C.inv_G2);
          } else if (mode == COL_RHS) {
            const float pk = pv[k1] * C.inv_G;
            b[k1] = cscale(make_float2(fmaf(-pk, b[k1].x, yv[k1].x), fmaf(-pk, b[k1].y, yv[k1].y)), C.inv_G);
          } else {  // COL_FWD
            zout[(size_t)j * G * G + kk] = cscale(b[k1], C.inv_G);
          }
        }
      }
      if (mode != COL_FWD) {
        dft<G1, true>(b);
#pragma unroll
        for (int m1 = 1; m1 < G1; ++m1) b[m1] = cmul(b[m1], twg<true>(C.tw, k2 * m1));
      }
    }
    if (mode == COL_FWD) {
      __syncthreads();
      continue;
    }
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int m1 = 0; m1 < G1; ++m1) sm[(m1 * G2 + k2) * TW + cc] = b[m1];
    }
    __syncthreads();
    STG(1, 2);
    {  // stage 3: thread (m1, c): inverse DFT over k2 -> y = m1 + G1 m2, keep y < N
      const int m1 = t / TW;
      if (m1 < G1 && colok) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = sm[(m1 * G2 + a2) * TW + (t % TW)];
        dft<G2, true>(d);
#pragma unroll
        for (int m2 = 0; m2 < K::B1; ++m2)
          if (in1<K>(m2, m1)) vio[((size_t)j * N + m1 + G1 * m2) * G + x] = d[m2];
      }
    }
    __syncthreads();
    STG(1, 3);
  }
}

// ------------------------------- D: row iFFT, channel products, W^-H along x
template <class K>
__device__ NLINV_PHASE void phase_row_d(const Ctx& C, float2* sm, const float2* rho, const float2* win,
                            float2* sout, float2* kbout) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, RS = K::RS;
  const int N = C.N, Gc = C.Gc, J = C.J;
  const int t = phase_tid();
  const int groups = (N + TW - 1) / TW;
  const int items = J * groups;
  for (int it = C.bid; it < items; it += C.nb) {
    const int j = it / groups;
    const int y0 = (it - j * groups) * TW;
    // stage-2 operands (c_j and rho rows) requested before stage 1 waits
    const int rr = t / G2, k2 = t % G2, y = y0 + rr;
    const bool ok = rr < TW && y < N;
    float2 cv[K::B2], rh[K::B2];
#pragma unroll
    for (int k1 = 0; k1 < K::B2; ++k1) {
      cv[k1] = rh[k1] = czero();
      if (ok && in2<K>(k1, k2)) {
        const int ir = y * N + k2 + G2 * k1;
        cv[k1] = ldcg(C.c + (size_t)j * N * N + ir);
        rh[k1] = ldcg(rho + ir);
      }
    }
    {  // stage 1: thread (row, n1): inverse DFT over n2
      const int r1 = t / G1, n1 = t % G1, y1 = y0 + r1;
      if (r1 < TW && y1 < N) {
        float2 a[G2];
        const float2* src = win + ((size_t)j * N + y1) * G;
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) a[n2] = ldcg(src + n1 + G1 * n2);
        dft<G2, true>(a);
#pragma unroll
        for (int q2 = 0; q2 < G2; ++q2) {
          float2 x = a[q2];
          if (q2) x = cmul(x, twg<true>(C.tw, n1 * q2));
          sm[r1 * RS + q2 * (G1 + 1) + n1] = x;
        }
      }
    }
    __syncthreads();
    // stage 2: thread (row, k2): inverse DFT over n1 -> t_j at x = k2 + G2 k1
    float2 g[G1];
    if (ok) {
      float2 b[G1];
#pragma unroll
      for (int n1 = 0; n1 < G1; ++n1) b[n1] = sm[rr * RS + k2 * (G1 + 1) + n1];
      dft<G1, true>(b);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1) {
        g[k1] = czero();
        if (k1 < K::B2 && in2<K>(k1, k2)) {
          const int kk = k1 < K::B2 ? k1 : 0;
          sout[((size_t)j * N + y) * N + k2 + G2 * k1] = cconjmul(cv[kk], b[k1]);
          g[k1] = cconjmul(rh[kk], b[k1]);
        }
      }
      dft<G1, false>(g);
#pragma unroll
      for (int kb = 1; kb < G1; ++kb) g[kb] = cmul(g[kb], twg<false>(C.tw, k2 * kb));
    }
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int kb = 0; kb < G1; ++kb) sm[rr * RS + kb * (G2 + 1) + k2] = g[kb];
    }
    __syncthreads();
    {  // stage 3: thread (row, kb): forward DFT over k2 -> kb + G1 ka, crop to G_c
      const int r3 = t / G1, kb = t % G1, y3 = y0 + r3;
      if (r3 < TW && y3 < N) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = sm[r3 * RS + kb * (G2 + 1) + a2];
        dft<G2, false>(d);
        float2* dst = kbout + ((size_t)j * N + y3) * Gc;
#pragma unroll
        for (int ka = 0; ka < G2; ++ka) {
          const int ix = coef_index(kb + G1 * ka, G, Gc);
          if (ix >= 0) dst[ix] = d[ka];
        }
      }
    }
    __syncthreads();
  }
}

// ----------------- E: W^-H along y, D_W^-1, channel sum, Tikhonov, Re<p,q>
// E_CG    : q = A p_k + alpha p_k (p_k in p_new), partial Re<p_k, q>
// E_RHS   : out = r = DF^H(...) - alpha (x_n - x_ref), partial |r|^2; hout = H r;
//           x_ref = xr_s * xr_in when xr_in is given (else the plan's x_ref)
// E_DFH   : out = DF^H z
// E_NORMAL: out = (DF^H P DF + alpha) dx                      (dx = p_new)
// E_CGR   : w = out = (DF^H P DF + alpha) r_k (r_k = p_new), partials of
//           Re<r_k, w> (slot) and |r_k|^2 (SLOT_RR0); hout = H w
// H is the y pass of W^-1 (as phase A computes it); for E_RHS and E_CGR the
// column values are still in registers, so it costs one more exchange.
template <class K, int mode>
__device__ NLINV_PHASE void phase_col_e(const Ctx& C, float2* sm, float2* sred, float alpha, int k,
                            const float2* kbin, const float2* sin, const float2* p_old,
                            float2* p_new, float2* out, float2* hout, int slot,
                            const float2* xr_in = nullptr, float xr_s = 1.f) {
  const float2* xr = xr_in ? xr_in : C.xref;   // E_RHS: regulariser xr_s * xr
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW;
  const int N = C.N, Gc = C.Gc, J = C.J, NN = N * N;
  const int t = phase_tid();
  const bool withH = (mode == E_RHS || mode == E_CGR);
  STG_BEGIN();
  const int tiles = (Gc + TW - 1) / TW;
  const int items = J * tiles;
  const Roles R = roles(C, items);
  float acc = 0.f;   // this thread's few terms; CTA and grid sums in float pairs
  float acc2 = 0.f;  // E_CGR: |r_k|^2
  if (R.items) for (int it = C.bid; it < items; it += R.istride) {
    const int j = it / tiles;
    const int fx = (it - j * tiles) * TW + (t % TW);
    const bool colok = fx < Gc;
    // every operand of the item is requested before anything waits: the
    // kb column (stage 1 mapping), then D_W^-1 and the CG / Tikhonov operands
    // of the kept rows (stage 2 mapping); beta's partials after them
    const int n1 = t / TW;
    float2 a[G2];
#pragma unroll
    for (int n2 = 0; n2 < G2; ++n2)
      a[n2] = (n1 < G1 && colok && in1<K>(n2, n1)) ? ldcg(kbin + ((size_t)j * N + n1 + G1 * n2) * Gc + fx)
                                                    : czero();
    const int k2 = t / TW, cc = t % TW;
    const bool ok = k2 < G2 && colok;
    float2 o1[G1], o2[G1];
    float dv[G1];
#pragma unroll
    for (int k1 = 0; k1 < G1; ++k1) {
      const int iy = coef_index(k2 + G2 * k1, G, Gc);
      o1[k1] = o2[k1] = czero();
      dv[k1] = 0.f;
      if (ok && iy >= 0) {
        const size_t e = (size_t)NN + ((size_t)j * Gc + iy) * Gc + fx;
        dv[k1] = __ldg(C.dinv + iy * Gc + fx);
        if (mode == E_CG || mode == E_NORMAL || mode == E_CGR) {
          o1[k1] = ldcg(p_new + e);
        } else if (mode == E_RHS) {
          o1[k1] = ldcg(C.xn + e);
          o2[k1] = ldcg(xr + e);
        }
      }
    }
    STG(2, 0);
    if (n1 < G1) {  // stage 1: thread (n1, c): forward DFT over n2 (rows y < N)
      dft<G2, false>(a);
#pragma unroll
      for (int q2 = 0; q2 < G2; ++q2) {
        float2 v = a[q2];
        if (q2) v = cmul(v, twg<false>(C.tw, n1 * q2));
        sm[(q2 * G1 + n1) * TW + (t % TW)] = v;
      }
    }
    __syncthreads();
    STG(2, 1);
    // stage 2: thread (k2, c): forward DFT over n1, crop rows to G_c, the
    // pointwise epilogue; then (E_RHS) D_W^-1 and the inverse DFT over k1 of
    // the new column for H
    float2 b[G1];
    if (ok) {
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = sm[(k2 * G1 + q1) * TW + cc];
      dft<G1, false>(b);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1) {
        const int iy = coef_index(k2 + G2 * k1, G, Gc);
        if (iy < 0) {
          b[k1] = czero();
          continue;
        }
        const size_t e = (size_t)NN + ((size_t)j * Gc + iy) * Gc + fx;
        const float2 val = cscale(b[k1], C.inv_G * dv[k1]);
        float2 res;
        if (mode == E_CG || mode == E_CGR) {
          res = cfma(o1[k1], alpha, val);
          acc = fmaf(o1[k1].x, res.x, fmaf(o1[k1].y, res.y, acc));
          if (mode == E_CGR) acc2 = fmaf(o1[k1].x, o1[k1].x, fmaf(o1[k1].y, o1[k1].y, acc2));
        } else if (mode == E_RHS) {
          res = cfma(cfma(o2[k1], -xr_s, o1[k1]), -alpha, val);
          acc = fmaf(res.x, res.x, fmaf(res.y, res.y, acc));
        } else if (mode == E_DFH) {
          res = val;
        } else {
          res = cfma(o1[k1], alpha, val);
        }
        out[e] = res;
        b[k1] = cscale(res, dv[k1]);
      }
      if (withH) {
        dft<G1, true>(b);
#pragma unroll
        for (int m1 = 1; m1 < G1; ++m1) b[m1] = cmul(b[m1], twg<true>(C.tw, k2 * m1));
      }
    }
    if (withH) {
      __syncthreads();
      if (ok) {
#pragma unroll
        for (int m1 = 0; m1 < G1; ++m1) sm[(m1 * G2 + k2) * TW + cc] = b[m1];
      }
      __syncthreads();
      {  // stage 3: thread (m1, c): inverse DFT over k2 -> y = m1 + G1 m2 < N
        const int m1 = t / TW;
        if (m1 < G1 && colok) {
          float2 d[G2];
#pragma unroll
          for (int a2 = 0; a2 < G2; ++a2) d[a2] = sm[(m1 * G2 + a2) * TW + (t % TW)];
          dft<G2, true>(d);
#pragma unroll
          for (int m2 = 0; m2 < K::B1; ++m2)
            if (in1<K>(m2, m1)) hout[((size_t)j * N + m1 + G1 * m2) * Gc + fx] = cscale(d[m2], C.inv_G);
        }
      }
    }
    __syncthreads();
  }
  STG(2, 2);
  // rho part: channel sum of s_j = conj(c_j) t_j (needs no CG scalar)
  if (R.elems) for (int e = R.ebid * blockDim.x + t; e < NN; e += R.enb * blockDim.x) {
    float2 o = czero(), o2v = czero();
    if (mode == E_CG || mode == E_NORMAL || mode == E_CGR) o = ldcg(p_new + e);
    if (mode == E_RHS) {
      o = ldcg(C.xn + e);
      o2v = ldcg(xr + e);
    }
    float2 sv = czero();
#pragma unroll 8
    for (int j = 0; j < J; ++j) sv = cadd(sv, ldcg(sin + (size_t)j * NN + e));
    if (mode == E_CG || mode == E_CGR) {
      const float2 qv = cfma(o, alpha, sv);
      out[e] = qv;
      acc = fmaf(o.x, qv.x, fmaf(o.y, qv.y, acc));
      if (mode == E_CGR) acc2 = fmaf(o.x, o.x, fmaf(o.y, o.y, acc2));
    } else if (mode == E_RHS) {
      const float2 bv = cfma(cfma(o2v, -xr_s, o), -alpha, sv);
      out[e] = bv;
      acc = fmaf(bv.x, bv.x, fmaf(bv.y, bv.y, acc));
    } else if (mode == E_DFH) {
      out[e] = sv;
    } else {
      out[e] = cfma(o, alpha, sv);
    }
  }
  STG(2, 3);
  if (mode == E_CG || mode == E_RHS || mode == E_CGR) block_partial(C, acc, slot, sred);
  if (mode == E_CGR) block_partial(C, acc2, SLOT_RR0, sred);
  STG(2, 4);
}

// -------------------------------------------------- F: CG vector update
// a = |r_k|^2 / Re<p_k, A p_k> (FP64); x += a p_k; r_{k+1} = r_k - a q;
// partial |r_{k+1}|^2; and H r_{k+1} (the y pass of W^-1 of the rounded new
// r) for the next direction.  r_k and r_{k+1} live in different buffers, so
// the column items (per channel and column tile, transform on chip) form
// r_{k+1} of their column in registers, exactly as the elementwise part
// stores it, while other CTAs already store r_{k+1}.  On the last iteration
// only x^_{n+1} = x^_n + x is applied.
template <class K>
__device__ NLINV_PHASE void phase_upd(const Ctx& C, float2* sm, float2* sred, int k, bool last,
                                       const float2* p) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW;
  constexpr int EU = NLINV_EU;   // elements per thread per round of the elementwise part
  const int N = C.N, Gc = C.Gc, J = C.J, NN = N * N;
  const int t = phase_tid();
  const float2* rk = C.rb[k & 1];
  float2* rk1 = C.rb[(k + 1) & 1];
  STG_BEGIN();
  __shared__ Scal2 s_a;
  Scal2 a{0.f, 0.f}, na{0.f, 0.f};
  bool need_a = true;
  // the step length, once per CTA and only after its first loads are issued
  auto get_a = [&]() {
    if (!need_a) return;
    need_a = false;
    if (t < 32) {
      const DF32 rrs = slot_sum(C, (k & 1) ? SLOT_RR1 : SLOT_RR0);
      const DF32 pqs = slot_sum(C, SLOT_PQ);
      if (t == 0) {
        const double rr = df_to_double(rrs);
        const double a64 = cg_step(rr, df_to_double(pqs));
        if (rr > 0.0 && a64 == 0.0) raise_err(C, DEV_ENUMERIC);
        const float hi = (float)a64;
        s_a = Scal2{hi, (float)(a64 - (double)hi)};
      }
    }
    __syncthreads();
    a = s_a;
    na = Scal2{-a.hi, -a.lo};
  };
  const int tiles = (Gc + TW - 1) / TW;
  const int items = last ? 0 : J * tiles;
  const Roles R = roles(C, items);
  float acc = 0.f;   // this thread's few terms; CTA and grid sums in float pairs
  // (1) H r_{k+1} per coil column tile
  if (R.items) for (int it = C.bid; it < items; it += R.istride) {
    const int j = it / tiles;
    const int fx = (it - j * tiles) * TW + (t % TW);
    const bool colok = fx < Gc;
    const int n1 = t / TW;
    float2 rv[G2], qv[G2];
    float dv[G2];
#pragma unroll
    for (int n2 = 0; n2 < G2; ++n2) {
      const int iy = coef_index(n1 + G1 * n2, G, Gc);
      rv[n2] = qv[n2] = czero();
      dv[n2] = 0.f;
      if (n1 < G1 && colok && iy >= 0) {
        const size_t e = (size_t)NN + ((size_t)j * Gc + iy) * Gc + fx;
        rv[n2] = ldcg(rk + e);
        qv[n2] = ldcg(C.q + e);
        dv[n2] = __ldg(C.dinv + iy * Gc + fx);
      }
    }
    get_a();
    STG(3, 0);
    if (n1 < G1) {  // stage 1: thread (n1, c): D_W^-1 r_{k+1} of the column, inverse DFT over n2
#pragma unroll
      for (int n2 = 0; n2 < G2; ++n2) rv[n2] = cscale(axpy2(qv[n2], na, rv[n2]), dv[n2]);
      dft<G2, true>(rv);
#pragma unroll
      for (int q2 = 0; q2 < G2; ++q2) {
        float2 x = rv[q2];
        if (q2) x = cmul(x, twg<true>(C.tw, n1 * q2));
        sm[(q2 * G1 + n1) * TW + (t % TW)] = x;
      }
    }
    __syncthreads();
    STG(3, 1);
    const int k2 = t / TW, cc = t % TW;
    if (k2 < G2 && colok) {  // stage 2: inverse DFT over n1, keep y < N
      float2 b[G1];
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = sm[(k2 * G1 + q1) * TW + cc];
      dft<G1, true>(b);
#pragma unroll
      for (int k1 = 0; k1 < K::B2; ++k1)
        if (in2<K>(k1, k2)) C.Hr[((size_t)j * N + k2 + G2 * k1) * Gc + fx] = cscale(b[k1], C.inv_G);
    }
    __syncthreads();
  }
  // (2) every element of x and r: a round's loads before the scalar and stores
  if (R.elems) {
    const int stride = R.enb * blockDim.x;
    for (int base = R.ebid * blockDim.x; base < C.nx; base += EU * stride) {   // CTA-uniform
      float2 pv[EU], qv[EU], rv[EU], xv[EU];
#pragma unroll
      for (int u = 0; u < EU; ++u) {
        const int e = base + t + u * stride;
        pv[u] = qv[u] = rv[u] = xv[u] = czero();
        if (e < C.nx) {
          pv[u] = ldcg(p + e);
          if (k > 0) xv[u] = ldcg(C.xcg + e);
          if (last) {
            rv[u] = ldcg(C.xn + e);
          } else {
            qv[u] = ldcg(C.q + e);
            rv[u] = ldcg(rk + e);
          }
        }
      }
      get_a();
#pragma unroll
      for (int u = 0; u < EU; ++u) {
        const int e = base + t + u * stride;
        if (e < C.nx) {
          const float2 xn = axpy2(pv[u], a, xv[u]);
          if (last) {
            C.xn[e] = cadd(rv[u], xn);
          } else {
            const float2 r1 = axpy2(qv[u], na, rv[u]);
            rk1[e] = r1;
            acc = fmaf(r1.x, r1.x, fmaf(r1.y, r1.y, acc));
            C.xcg[e] = xn;
          }
        }
      }
    }
  }
  STG(3, 2);
  if (!last) block_partial(C, acc, (k & 1) ? SLOT_RR0 : SLOT_RR1, sred);
  STG(3, 4);
}

// x^_0 = x_prev (or rho = 1, c^ = 0), x_ref = damping * x_prev
__device__ __forceinline__ void phase_init(const Ctx& C, const float2* xprev, float damping) {
  const int NN = C.N * C.N;
  for (int e = C.bid * blockDim.x + threadIdx.x; e < C.nx; e += C.nb * blockDim.x) {
    float2 v = xprev ? ldcg(xprev + e) : make_float2(e < NN ? 1.f : 0.f, 0.f);
    C.xn[e] = v;
    C.xref[e] = cscale(v, damping);
  }
}

// outputs: x^ copy, rho, rho * sqrt(sum_j |c_j|^2)
__device__ __forceinline__ void phase_final(const Ctx& C, float2* xout, float2* rho_out, float2* img_out) {
  const int NN = C.N * C.N;
  for (int e = C.bid * blockDim.x + threadIdx.x; e < C.nx; e += C.nb * blockDim.x) {
    const float2 v = ldcg(C.xn + e);
    if (xout) xout[e] = v;
    if (e < NN) {
      if (rho_out) rho_out[e] = v;
      if (img_out) {
        float ss = 0.f;
        for (int j = 0; j < C.J; ++j) {
          const float2 cv = ldcg(C.c + (size_t)j * NN + e);
          ss = fmaf(cv.x, cv.x, fmaf(cv.y, cv.y, ss));
        }
        img_out[e] = cscale(v, sqrtf(ss));
      }
    }
  }
}

// ------------------------------------------------------- grid barrier
// Monotone-counter barrier of the CTAs working on one frame (the whole grid,
// or one frame group of a batch launch): arrival is an acq_rel atomic add on
// the group's counter (zeroed before each launch); barrier number e is passed
// once the counter reaches e * nb.  Every wait is
// bounded by spin_limit polls; on expiry the error word is set and all CTAs
// leave at their next barrier.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned o;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(o) : "l"(p), "r"(v) : "memory");
  return o;
}

__device__ __forceinline__ bool grid_sync(const Ctx& C, unsigned& epoch) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned target = epoch * (unsigned)C.nb;
    const unsigned prev = atom_add_acq_rel(C.bar, 1u);
    if (prev + 1 != target) {
      long long it = 0;
      while ((int)(ld_acquire(C.bar) - target) < 0) {
        if (*(volatile int*)C.err != 0) break;
        if (++it > C.spin_limit) {
          raise_err(C, DEV_ETIMEOUT);
          break;
        }
        if (NLINV_BAR_SLEEP_NS > 0) __nanosleep(NLINV_BAR_SLEEP_NS);
      }
    }
  }
  __syncthreads();
  return *(volatile int*)C.err == 0;
}

}  // namespace nlinv
