// Cluster-resident phases of the NLINV frame (Schaetz et al. 2017, Sec. 2.2,
// Eqs. (2)-(5), Fig. 4) for one GB300.
//
// One thread-block cluster of CS CTAs owns one receive channel j.  The
// channel's per-phase data never goes through L2: CTA `rank` of the cluster
// owns image rows [rank R, rank R + R) for the row passes and grid columns
// [rank C, rank C + C) (coil columns [rank Cc, rank Cc + Cc)) for the column
// passes, and a pass stores each result straight into the shared memory of
// the CTA that owns it in the next pass (st.shared::cluster to the address
// mapa gives), so the transposes between row and column passes are
// distributed-shared-memory pushes followed by a cluster barrier.  Only the
// channel sum sum_j conj(c_j) t_j and the two CG inner products couple the
// channels; they meet at the two grid barriers of a CG iteration.
//
// Shared memory of a CTA (float2 unless noted):
//   RB  [R][RS]   rows of the current row pass; also the row FFT's exchange
//   CB  [N][C]    this CTA's columns of the row pass output
//   XB  [G][TW]   exchange of the column FFT (TW columns at a time)
//   HB  [R][Gc]   rows of H = y pass of W^-1 (coil band of the row)
//   KB  [N][Cc]   this CTA's coil columns of the W^-H x pass
//   CJ  [R][N]    coil map rows c_j of the Newton step's linearisation point
//   VO  [N][C]    T(p_{k-1}) of this CTA's columns (CG direction recurrence)
// The unknowns and the CG vectors (rho part and coil part) stay in global
// memory: the rho part is updated elementwise by all CTAs, the coil part of
// channel j only by the CTAs of cluster j, each on its own coil columns.
#pragma once
#include "phases.cuh"

namespace nlinv {
namespace cl {

__device__ __forceinline__ unsigned ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// the address of the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ unsigned remote(unsigned local, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_remote(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void csync() {
  arrive();
  wait();
}

// Partition and shared-memory layout of the cluster kernel (host-computed).
struct Lay {
  int CS;                     // CTAs per cluster (one cluster per channel)
  int R, C, Cc;               // rows / grid columns / coil columns per CTA
  int rb, cb, xb, hb, kb, cj, vo;   // float2 offsets in dynamic shared memory
  int smem_bytes;
};

// Per-CTA view: the channel, the rank, the partition bounds and the shared
// buffers (local pointers and their shared-window addresses for pushes).
struct View {
  int j, rank;
  int y0, ny;                 // rows [y0, y0 + ny)
  int x0, nxc;                // grid columns [x0, x0 + nxc)
  int f0, nf;                 // coil columns [f0, f0 + nf)
  float2 *rb, *cb, *xb, *hb, *kb, *cj, *vo;
  unsigned a_rb, a_cb, a_hb, a_kb;
};

// Built at the start of every phase (nothing of it stays live across the
// persistent kernel's phases): the rank comes from an opaque read.
template <class K>
__device__ __forceinline__ View make_view(const Ctx& C, const Lay& L, float2* sm) {
  View v;
  v.j = blockIdx.x / L.CS;
  v.rank = (int)ctarank();
  const int N = K::NR, G = K::G;
  v.y0 = v.rank * L.R;
  v.ny = max(0, min(L.R, N - v.y0));
  v.x0 = v.rank * L.C;
  v.nxc = max(0, min(L.C, G - v.x0));
  v.f0 = v.rank * L.Cc;
  v.nf = max(0, min(L.Cc, C.Gc - v.f0));
  v.rb = sm + L.rb;
  v.cb = sm + L.cb;
  v.xb = sm + L.xb;
  v.hb = sm + L.hb;
  v.kb = sm + L.kb;
  v.cj = sm + L.cj;
  v.vo = sm + L.vo;
  v.a_rb = saddr(v.rb);
  v.a_cb = saddr(v.cb);
  v.a_hb = saddr(v.hb);
  v.a_kb = saddr(v.kb);
  return v;
}

// ------------------------------------------------------------ pushes
// element (y, x) of a row pass output -> CB[y][x - owner C] of the owner of x
__device__ __forceinline__ void push_cb(const Lay& L, const View& v, int y, int x, float2 val) {
  const int o = x / L.C;
  st_remote(remote(v.a_cb + 8u * (unsigned)(y * L.C + (x - o * L.C)), o), val);
}
// element (y, x) of a column pass output -> RB[y - owner R][x] of the owner of y
template <class K>
__device__ __forceinline__ void push_rb(const Lay& L, const View& v, int y, int x, float2 val) {
  const int o = y / L.R;
  st_remote(remote(v.a_rb + 8u * (unsigned)((y - o * L.R) * K::RS + x), o), val);
}
// element (y, fx) of a coil column pass output (H) -> HB[y - owner R][fx]
__device__ __forceinline__ void push_hb(const Lay& L, const View& v, int Gc, int y, int fx, float2 val) {
  const int o = y / L.R;
  st_remote(remote(v.a_hb + 8u * (unsigned)((y - o * L.R) * Gc + fx), o), val);
}
// element (y, coil index ix) of the W^-H x pass -> KB[y][ix - owner Cc]
__device__ __forceinline__ void push_kb(const Lay& L, const View& v, int y, int ix, float2 val) {
  const int o = ix / L.Cc;
  st_remote(remote(v.a_kb + 8u * (unsigned)(y * L.Cc + (ix - o * L.Cc)), o), val);
}

// ------------------------------------------ coil column pass: H = W^-1 along y
// H(src) of this CTA's coil columns: D_W^-1, inverse DFT along y (Gc nonzero
// of G), keep rows y < N, 1/G; pushed to HB of the row owners.
// src: coil part [J][Gc][Gc] of a vector (global).
template <class K>
__device__ __forceinline__ void coil_y(const Ctx& C, const Lay& L, float2* sm, const float2* src) {
  const View v = make_view<K>(C, L, sm);
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW;
  const int Gc = C.Gc, j = v.j;
  const int t = phase_tid();
  for (int c0 = 0; c0 < v.nf; c0 += TW) {
    const int cc = t % TW;
    const int fx = v.f0 + c0 + cc;
    const bool colok = c0 + cc < v.nf;
    {
      const int n1 = t / TW;
      if (n1 < G1) {
        float2 a[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          const int iy = coef_index(n1 + G1 * n2, G, Gc);
          a[n2] = (colok && iy >= 0) ? cscale(ldcg(src + ((size_t)j * Gc + iy) * Gc + fx), __ldg(C.dinv + iy * Gc + fx))
                                     : czero();
        }
        dft<G2, true>(a);
#pragma unroll
        for (int k2 = 0; k2 < G2; ++k2) {
          float2 x = a[k2];
          if (k2) x = cmul(x, twg<true>(C.tw, n1 * k2));
          v.xb[(k2 * G1 + n1) * TW + cc] = x;
        }
      }
    }
    __syncthreads();
    {
      const int k2 = t / TW;
      if (k2 < G2 && colok) {
        float2 b[G1];
#pragma unroll
        for (int n1 = 0; n1 < G1; ++n1) b[n1] = v.xb[(k2 * G1 + n1) * TW + cc];
        dft<G1, true>(b);
#pragma unroll
        for (int k1 = 0; k1 < K::B2; ++k1)
          if (in2<K>(k1, k2)) push_hb(L, v, Gc, k2 + G2 * k1, fx, cscale(b[k1], C.inv_G));
      }
    }
    __syncthreads();
  }
}

// --------------------------------------------- row pass B (Newton step set-up)
// ROW_COIL: c_j = W^-1 c^_j of the rows (kept in CJ and in the global coil
// maps), u = rho c_j, forward FFT of the padded row, pushed to CB.
// ROW_COILONLY: the coil maps only (global), for the final image.
template <class K>
__device__ __forceinline__ void row_b(const Ctx& C, const Lay& L, float2* sm, int mode) {
  const View v = make_view<K>(C, L, sm);
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, RS = K::RS, N = K::NR;
  const int Gc = C.Gc, j = v.j;
  const int t = phase_tid();
  for (int r0 = 0; r0 < v.ny; r0 += TW) {
    {  // stage 1: thread (row, n1): inverse DFT over n2 of the coil band
      const int rr = t / G1, n1 = t % G1;
      if (rr < TW && r0 + rr < v.ny) {
        float2 a[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          const int ix = coef_index(n1 + G1 * n2, G, Gc);
          a[n2] = ix >= 0 ? v.hb[(r0 + rr) * Gc + ix] : czero();
        }
        dft<G2, true>(a);
#pragma unroll
        for (int k2 = 0; k2 < G2; ++k2) {
          float2 x = a[k2];
          if (k2) x = cmul(x, twg<true>(C.tw, n1 * k2));
          v.rb[(r0 + rr) * RS + k2 * (G1 + 1) + n1] = x;
        }
      }
    }
    __syncthreads();
    const int rr = t / G2, k2 = t % G2;
    const bool ok = rr < TW && r0 + rr < v.ny;
    const int yl = r0 + rr, y = v.y0 + yl;
    float2 u[G1];
    if (ok) {
      float2 b[G1];
#pragma unroll
      for (int n1 = 0; n1 < G1; ++n1) b[n1] = v.rb[yl * RS + k2 * (G1 + 1) + n1];
      dft<G1, true>(b);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1) {
        u[k1] = czero();
        if (in2<K>(k1, k2)) {
          const int x = k2 + G2 * k1;
          C.c[((size_t)j * N + y) * N + x] = b[k1];
          if (mode == ROW_COIL) {
            v.cj[yl * N + x] = b[k1];
            u[k1] = cmul(ldcg(C.xn + y * N + x), b[k1]);
          }
        }
      }
      if (mode == ROW_COIL) {
        dft<G1, false>(u);
#pragma unroll
        for (int kb = 1; kb < G1; ++kb) u[kb] = cmul(u[kb], twg<false>(C.tw, k2 * kb));
      }
    }
    __syncthreads();
    if (mode != ROW_COIL) continue;
    if (ok) {
#pragma unroll
      for (int kb = 0; kb < G1; ++kb) v.rb[yl * RS + kb * (G2 + 1) + k2] = u[kb];
    }
    __syncthreads();
    {  // stage 3: thread (row, kb): forward DFT over k2 -> x = kb + G1 ka, pushed
      const int r3 = t / G1, kb = t % G1;
      if (r3 < TW && r0 + r3 < v.ny) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = v.rb[(r0 + r3) * RS + kb * (G2 + 1) + a2];
        dft<G2, false>(d);
        const int y3 = v.y0 + r0 + r3;
#pragma unroll
        for (int ka = 0; ka < G2; ++ka) push_cb(L, v, y3, kb + G1 * ka, d[ka]);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------- row pass of a CG iteration: T(r_k)
// x pass of W^-1 of H r_k (HB), u = c_j r_rho + rho dc, forward row FFT,
// pushed to CB.  rk: the residual (global; its rho part is read).
template <class K>
__device__ __forceinline__ void row_cg(const Ctx& C, const Lay& L, float2* sm, const float2* rk) {
  const View v = make_view<K>(C, L, sm);
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, RS = K::RS, N = K::NR;
  const int Gc = C.Gc;
  const int t = phase_tid();
  for (int r0 = 0; r0 < v.ny; r0 += TW) {
    const int rr = t / G2, k2 = t % G2;
    const bool ok = rr < TW && r0 + rr < v.ny;
    const int yl = r0 + rr, y = v.y0 + yl;
    float2 rv[K::B2], rh[K::B2];   // stage-2 operands requested before stage 1
#pragma unroll
    for (int k1 = 0; k1 < K::B2; ++k1) {
      rv[k1] = rh[k1] = czero();
      if (ok && in2<K>(k1, k2)) {
        const int ir = y * N + k2 + G2 * k1;
        rv[k1] = ldcg(rk + ir);
        rh[k1] = ldcg(C.xn + ir);
      }
    }
    {
      const int r1 = t / G1, n1 = t % G1;
      if (r1 < TW && r0 + r1 < v.ny) {
        float2 a[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          const int ix = coef_index(n1 + G1 * n2, G, Gc);
          a[n2] = ix >= 0 ? v.hb[(r0 + r1) * Gc + ix] : czero();
        }
        dft<G2, true>(a);
#pragma unroll
        for (int q2 = 0; q2 < G2; ++q2) {
          float2 x = a[q2];
          if (q2) x = cmul(x, twg<true>(C.tw, n1 * q2));
          v.rb[(r0 + r1) * RS + q2 * (G1 + 1) + n1] = x;
        }
      }
    }
    __syncthreads();
    float2 u[G1];
    if (ok) {
      float2 b[G1];
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = v.rb[yl * RS + k2 * (G1 + 1) + q1];
      dft<G1, true>(b);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1)
        u[k1] = (k1 < K::B2 && in2<K>(k1, k2))
                    ? cadd(cmul(v.cj[yl * N + k2 + G2 * k1], rv[k1 < K::B2 ? k1 : 0]), cmul(rh[k1 < K::B2 ? k1 : 0], b[k1]))
                    : czero();
      dft<G1, false>(u);
#pragma unroll
      for (int kb = 1; kb < G1; ++kb) u[kb] = cmul(u[kb], twg<false>(C.tw, k2 * kb));
    }
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int kb = 0; kb < G1; ++kb) v.rb[yl * RS + kb * (G2 + 1) + k2] = u[kb];
    }
    __syncthreads();
    {
      const int r3 = t / G1, kb = t % G1;
      if (r3 < TW && r0 + r3 < v.ny) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = v.rb[(r0 + r3) * RS + kb * (G2 + 1) + a2];
        dft<G2, false>(d);
        const int y3 = v.y0 + r0 + r3;
#pragma unroll
        for (int ka = 0; ka < G2; ++ka) push_cb(L, v, y3, kb + G1 * ka, d[ka]);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------ column pass (PSF)
// COL_CG  : T(p_k) = CB + beta VO (kept in VO), then as COL_TOEP
// COL_TOEP: FFT_y, x P / G^2, iFFT_y, keep N rows
// COL_RHS : FFT_y, (Y - P X / G) / G, iFFT_y, keep N rows
// The kept rows are pushed to RB of their row owners.
template <class K>
__device__ __forceinline__ void col_c(const Ctx& C, const Lay& L, float2* sm, int mode, const float* P,
                                      const float2* Yin, Scal2 beta, bool first) {
  const View v = make_view<K>(C, L, sm);
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW;
  const int j = v.j;
  const int t = phase_tid();
  const bool cg = (mode == COL_CG);
  for (int c0 = 0; c0 < v.nxc; c0 += TW) {
    const int cc = t % TW;
    const int xl = c0 + cc, x = v.x0 + xl;
    const bool colok = xl < v.nxc;
    const int k2 = t / TW;
    const bool ok = k2 < G2 && colok;
    float pv[G1];
    float2 yv[G1];
#pragma unroll
    for (int k1 = 0; k1 < G1; ++k1) {
      const size_t kk = (size_t)(k2 + G2 * k1) * G + x;
      pv[k1] = ok ? __ldg(P + kk) : 0.f;
      yv[k1] = (ok && mode == COL_RHS) ? ldcg(Yin + (size_t)j * G * G + kk) : czero();
    }
    {  // stage 1: thread (n1, c): forward DFT over n2 (rows y = n1 + G1 n2 < N)
      const int n1 = t / TW;
      if (n1 < G1 && colok) {
        float2 a[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          a[n2] = czero();
          if (in1<K>(n2, n1)) {
            const int y = n1 + G1 * n2;
            a[n2] = v.cb[y * L.C + xl];
            if (cg) {
              if (!first) a[n2] = axpy2(v.vo[y * L.C + xl], beta, a[n2]);
              v.vo[y * L.C + xl] = a[n2];
            }
          }
        }
        dft<G2, false>(a);
#pragma unroll
        for (int q2 = 0; q2 < G2; ++q2) {
          float2 w = a[q2];
          if (q2) w = cmul(w, twg<false>(C.tw, n1 * q2));
          v.xb[(q2 * G1 + n1) * TW + cc] = w;
        }
      }
    }
    __syncthreads();
    float2 b[G1];
    if (ok) {
#pragma unroll
      for (int n1 = 0; n1 < G1; ++n1) b[n1] = v.xb[(k2 * G1 + n1) * TW + cc];
      dft<G1, false>(b);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1) {
        if (mode == COL_RHS) {
          const float pk = pv[k1] * C.inv_G;
          b[k1] = cscale(make_float2(fmaf(-pk, b[k1].x, yv[k1].x), fmaf(-pk, b[k1].y, yv[k1].y)), C.inv_G);
        } else {
          b[k1] = cscale(b[k1], pv[k1] * C.inv_G2);
        }
      }
      dft<G1, true>(b);
#pragma unroll
      for (int m1 = 1; m1 < G1; ++m1) b[m1] = cmul(b[m1], twg<true>(C.tw, k2 * m1));
    }
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int m1 = 0; m1 < G1; ++m1) v.xb[(m1 * G2 + k2) * TW + cc] = b[m1];
    }
    __syncthreads();
    {  // stage 3: thread (m1, c): inverse DFT over k2 -> y = m1 + G1 m2 < N, pushed
      const int m1 = t / TW;
      if (m1 < G1 && colok) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = v.xb[(m1 * G2 + a2) * TW + cc];
        dft<G2, true>(d);
#pragma unroll
        for (int m2 = 0; m2 < K::B1; ++m2)
          if (in1<K>(m2, m1)) push_rb<K>(L, v, m1 + G1 * m2, x, d[m2]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------- row pass D: t_j, channel products, W^-H along x
// t_j = iFFT_x of the RB rows (keep N); s_j = conj(c_j) t_j to the global
// channel-sum buffer; conj(rho) t_j forward FFT'd along x, cropped to the
// coil band and pushed to KB.  When pr is given (a CG iteration), the thread
// also accumulates Re<p_rho, s_j> with p_rho = r_rho + beta p_old_rho formed
// on the fly (pq: the caller's running term of Re<p, A p>).
template <class K>
__device__ __forceinline__ void row_d(const Ctx& C, const Lay& L, float2* sm, const float2* pr_r,
                                      const float2* pr_old, Scal2 beta, bool first, float& pq) {
  const View v = make_view<K>(C, L, sm);
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, RS = K::RS, N = K::NR;
  const int Gc = C.Gc, j = v.j;
  const int t = phase_tid();
  for (int r0 = 0; r0 < v.ny; r0 += TW) {
    const int rr = t / G2, k2 = t % G2;
    const bool ok = rr < TW && r0 + rr < v.ny;
    const int yl = r0 + rr, y = v.y0 + yl;
    float2 rh[K::B2], pp[K::B2];
#pragma unroll
    for (int k1 = 0; k1 < K::B2; ++k1) {
      rh[k1] = pp[k1] = czero();
      if (ok && in2<K>(k1, k2)) {
        const int ir = y * N + k2 + G2 * k1;
        rh[k1] = ldcg(C.xn + ir);
        if (pr_r) {
          pp[k1] = ldcg(pr_r + ir);
          if (!first) pp[k1] = axpy2(ldcg(pr_old + ir), beta, pp[k1]);
        }
      }
    }
    float2 a[G2];
    const int r1 = t / G1, n1 = t % G1;
    const bool ok1 = r1 < TW && r0 + r1 < v.ny;
    if (ok1) {
#pragma unroll
      for (int n2 = 0; n2 < G2; ++n2) a[n2] = v.rb[(r0 + r1) * RS + n1 + G1 * n2];
    }
    __syncthreads();   // every row element read before the exchange overwrites it
    if (ok1) {
      dft<G2, true>(a);
#pragma unroll
      for (int q2 = 0; q2 < G2; ++q2) {
        float2 x = a[q2];
        if (q2) x = cmul(x, twg<true>(C.tw, n1 * q2));
        v.rb[(r0 + r1) * RS + q2 * (G1 + 1) + n1] = x;
      }
    }
    __syncthreads();
    float2 g[G1];
    if (ok) {
      float2 b[G1];
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = v.rb[yl * RS + k2 * (G1 + 1) + q1];
      dft<G1, true>(b);
#pragma unroll
      for (int k1 = 0; k1 < G1; ++k1) {
        g[k1] = czero();
        if (k1 < K::B2 && in2<K>(k1, k2)) {
          const int kk = k1 < K::B2 ? k1 : 0;
          const int x = k2 + G2 * k1;
          const float2 sv = cconjmul(v.cj[yl * N + x], b[k1]);
          C.s[((size_t)j * N + y) * N + x] = sv;
          if (pr_r) pq = fmaf(pp[kk].x, sv.x, fmaf(pp[kk].y, sv.y, pq));
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
      for (int kb = 0; kb < G1; ++kb) v.rb[yl * RS + kb * (G2 + 1) + k2] = g[kb];
    }
    __syncthreads();
    {
      const int r3 = t / G1, kb = t % G1;
      if (r3 < TW && r0 + r3 < v.ny) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = v.rb[(r0 + r3) * RS + kb * (G2 + 1) + a2];
        dft<G2, false>(d);
        const int y3 = v.y0 + r0 + r3;
#pragma unroll
        for (int ka = 0; ka < G2; ++ka) {
          const int ix = coef_index(kb + G1 * ka, G, Gc);
          if (ix >= 0) push_kb(L, v, y3, ix, d[ka]);
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------- coil column pass E: W^-H along y
// E_CG : p_c = r_c + beta p_old_c of the columns (stored to p_new), q_c = A p
//        + alpha p_c (to C.q), pq += Re<p_c, q_c>
// E_RHS: r_0c = DF^H(...)_c - alpha (x_c - xr_s x_ref_c) (to out), rr +=
//        |r_0c|^2, and H r_0 pushed to HB
template <class K, int mode>
__device__ __forceinline__ void col_e(const Ctx& C, const Lay& L, float2* sm, float alpha, Scal2 beta,
                                      bool first, const float2* r_c, const float2* p_old, float2* p_new,
                                      float2* out, const float2* xr, float xr_s, float& acc) {
  const View v = make_view<K>(C, L, sm);
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, N = K::NR;
  const int Gc = C.Gc, j = v.j, NN = N * N;
  const int t = phase_tid();
  for (int c0 = 0; c0 < v.nf; c0 += TW) {
    const int cc = t % TW;
    const int fl = c0 + cc, fx = v.f0 + fl;
    const bool colok = fl < v.nf;
    const int n1 = t / TW;
    float2 a[G2];
#pragma unroll
    for (int n2 = 0; n2 < G2; ++n2)
      a[n2] = (n1 < G1 && colok && in1<K>(n2, n1)) ? v.kb[(n1 + G1 * n2) * L.Cc + fl] : czero();
    const int k2 = t / TW;
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
        if (mode == E_CG) {
          o1[k1] = ldcg(r_c + e);
          if (!first) o1[k1] = axpy2(ldcg(p_old + e), beta, o1[k1]);
        } else {
          o1[k1] = ldcg(C.xn + e);
          o2[k1] = ldcg(xr + e);
        }
      }
    }
    if (n1 < G1) {
      dft<G2, false>(a);
#pragma unroll
      for (int q2 = 0; q2 < G2; ++q2) {
        float2 w = a[q2];
        if (q2) w = cmul(w, twg<false>(C.tw, n1 * q2));
        v.xb[(q2 * G1 + n1) * TW + cc] = w;
      }
    }
    __syncthreads();
    float2 b[G1];
    if (ok) {
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = v.xb[(k2 * G1 + q1) * TW + cc];
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
        if (mode == E_CG) {
          p_new[e] = o1[k1];
          const float2 q = cfma(o1[k1], alpha, val);
          C.q[e] = q;
          acc = fmaf(o1[k1].x, q.x, fmaf(o1[k1].y, q.y, acc));
        } else {
          const float2 res = cfma(cfma(o2[k1], -xr_s, o1[k1]), -alpha, val);
          out[e] = res;
          acc = fmaf(res.x, res.x, fmaf(res.y, res.y, acc));
          b[k1] = cscale(res, dv[k1]);
        }
      }
      if (mode == E_RHS) {
        dft<G1, true>(b);
#pragma unroll
        for (int m1 = 1; m1 < G1; ++m1) b[m1] = cmul(b[m1], twg<true>(C.tw, k2 * m1));
      }
    }
    if (mode == E_RHS) {
      __syncthreads();
      if (ok) {
#pragma unroll
        for (int m1 = 0; m1 < G1; ++m1) v.xb[(m1 * G2 + k2) * TW + cc] = b[m1];
      }
      __syncthreads();
      const int m1 = t / TW;
      if (m1 < G1 && colok) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = v.xb[(m1 * G2 + a2) * TW + cc];
        dft<G2, true>(d);
#pragma unroll
        for (int m2 = 0; m2 < K::B1; ++m2)
          if (in1<K>(m2, m1)) push_hb(L, v, Gc, m1 + G1 * m2, fx, cscale(d[m2], C.inv_G));
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------- coil columns of the update
// r_{k+1,c} = r_c - a q_c (to r1), x_cg,c (+)= a p_c, rr += |r_{k+1,c}|^2,
// H r_{k+1} pushed to HB; on the last iteration x^_{n+1,c} = x^_{n,c} +
// x_cg,c + a p_c instead.
template <class K>
__device__ __forceinline__ void upd_coil(const Ctx& C, const Lay& L, float2* sm, Scal2 a, bool first, bool last,
                                         const float2* rk, float2* rk1, const float2* p, float& acc) {
  const View v = make_view<K>(C, L, sm);
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, N = K::NR;
  const int Gc = C.Gc, j = v.j, NN = N * N;
  const int t = phase_tid();
  const Scal2 na{-a.hi, -a.lo};
  for (int c0 = 0; c0 < v.nf; c0 += TW) {
    const int cc = t % TW;
    const int fl = c0 + cc, fx = v.f0 + fl;
    const bool colok = fl < v.nf;
    const int n1 = t / TW;
    float2 rv[G2];
#pragma unroll
    for (int n2 = 0; n2 < G2; ++n2) {
      rv[n2] = czero();
      const int iy = coef_index(n1 + G1 * n2, G, Gc);
      if (n1 < G1 && colok && iy >= 0) {
        const size_t e = (size_t)NN + ((size_t)j * Gc + iy) * Gc + fx;
        const float2 pv = ldcg(p + e);
        const float2 xv = first ? czero() : ldcg(C.xcg + e);
        const float2 xs = axpy2(pv, a, xv);
        if (last) {
          C.xn[e] = cadd(ldcg(C.xn + e), xs);
        } else {
          C.xcg[e] = xs;
          const float2 r1 = axpy2(ldcg(C.q + e), na, ldcg(rk + e));
          rk1[e] = r1;
          acc = fmaf(r1.x, r1.x, fmaf(r1.y, r1.y, acc));
          rv[n2] = cscale(r1, __ldg(C.dinv + iy * Gc + fx));
        }
      }
    }
    if (last) continue;   // uniform over the CTA
    if (n1 < G1) {
      dft<G2, true>(rv);
#pragma unroll
      for (int q2 = 0; q2 < G2; ++q2) {
        float2 w = rv[q2];
        if (q2) w = cmul(w, twg<true>(C.tw, n1 * q2));
        v.xb[(q2 * G1 + n1) * TW + cc] = w;
      }
    }
    __syncthreads();
    const int k2 = t / TW;
    if (k2 < G2 && colok) {
      float2 b[G1];
#pragma unroll
      for (int q1 = 0; q1 < G1; ++q1) b[q1] = v.xb[(k2 * G1 + q1) * TW + cc];
      dft<G1, true>(b);
#pragma unroll
      for (int k1 = 0; k1 < K::B2; ++k1)
        if (in2<K>(k1, k2)) push_hb(L, v, Gc, k2 + G2 * k1, fx, cscale(b[k1], C.inv_G));
    }
    __syncthreads();
  }
}

// ---------------------------------------------- rho part (all CTAs, elementwise)
// The image part of every vector is split over all CTAs of the launch in
// contiguous slices; these run between the grid barriers.

// r_0,rho = sum_j s_j - alpha (x_rho - xr_s x_ref_rho); rr += |r_0,rho|^2
__device__ __forceinline__ void rho_rhs(const Ctx& C, float alpha, const float2* xr, float xr_s, float& acc) {
  const int NN = C.N * C.N, J = C.J;
  const int t = phase_tid();
  for (int e = C.bid * blockDim.x + t; e < NN; e += C.nb * blockDim.x) {
    const float2 xo = ldcg(C.xn + e), xv = ldcg(xr + e);
    float2 sv = czero();
#pragma unroll 8
    for (int j = 0; j < J; ++j) sv = cadd(sv, ldcg(C.s + (size_t)j * NN + e));
    const float2 b = cfma(cfma(xv, -xr_s, xo), -alpha, sv);
    C.rb[0][e] = b;
    acc = fmaf(b.x, b.x, fmaf(b.y, b.y, acc));
  }
}

// p_k,rho = r_k,rho + beta p_{k-1},rho (p_0 = r_0); pq += alpha |p_k,rho|^2
__device__ __forceinline__ void rho_p(const Ctx& C, const float2* rk, const float2* p_old, float2* p_new,
                                      Scal2 beta, bool first, float alpha, float& acc) {
  const int NN = C.N * C.N;
  const int t = phase_tid();
  for (int e = C.bid * blockDim.x + t; e < NN; e += C.nb * blockDim.x) {
    float2 pv = ldcg(rk + e);
    if (!first) pv = axpy2(ldcg(p_old + e), beta, pv);
    p_new[e] = pv;
    acc = fmaf(alpha * pv.x, pv.x, fmaf(alpha * pv.y, pv.y, acc));
  }
}

// q_rho = sum_j s_j + alpha p_rho; x_cg,rho (+)= a p_rho; r_{k+1},rho =
// r_rho - a q_rho, rr += |r_{k+1},rho|^2; on the last iteration x^_{n+1},rho
// = x^_n,rho + x_cg,rho + a p_rho instead.
__device__ __forceinline__ void rho_upd(const Ctx& C, Scal2 a, bool first, bool last, float alpha,
                                        const float2* rk, float2* rk1, const float2* p, float& acc) {
  const int NN = C.N * C.N, J = C.J;
  const int t = phase_tid();
  const Scal2 na{-a.hi, -a.lo};
  for (int e = C.bid * blockDim.x + t; e < NN; e += C.nb * blockDim.x) {
    const float2 pv = ldcg(p + e);
    const float2 xv = first ? czero() : ldcg(C.xcg + e);
    const float2 xs = axpy2(pv, a, xv);
    if (last) {
      C.xn[e] = cadd(ldcg(C.xn + e), xs);
      continue;
    }
    C.xcg[e] = xs;
    float2 sv = czero();
#pragma unroll 8
    for (int j = 0; j < J; ++j) sv = cadd(sv, ldcg(C.s + (size_t)j * NN + e));
    const float2 q = cfma(pv, alpha, sv);
    const float2 r1 = axpy2(q, na, ldcg(rk + e));
    rk1[e] = r1;
    acc = fmaf(r1.x, r1.x, fmaf(r1.y, r1.y, acc));
  }
}

}  // namespace cl
}  // namespace nlinv
