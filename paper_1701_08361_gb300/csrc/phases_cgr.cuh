// The CG of the per-phase path with the operator applied to the residual
// (Sec. 2.2, Eq. (4): the same Krylov iterates as the textbook CG in exact
// arithmetic, in the arrangement of Chronopoulos and Gear, 1989).  With
// w_k = A r_k the step lengths follow from gamma_k = |r_k|^2 and
// delta_k = Re<r_k, w_k>, which one column pass forms together:
//   beta_k = gamma_k / gamma_{k-1}            (beta_0 = 0)
//   a_k    = gamma_k / (delta_k - beta_k gamma_k / a_{k-1})
//   p_k = r_k + beta_k p_{k-1},  s_k = w_k + beta_k s_{k-1}   (s_k = A p_k)
//   x_{k+1} = x_k + a_k p_k,     r_{k+1} = r_k - a_k s_k
// so a CG iteration is four phases -- the row pass of r_k (which also applies
// the previous step's vector update), the PSF column pass, the row pass back
// with the channel products, and the W^-H column pass that forms w_k, its two
// inner products and H w_k -- and one reduction point instead of two.
#pragma once
#include "phases.cuh"

namespace nlinv {

// slot_sum of two slots in one pass: both slots' loads are issued before
// any add (one L2 round trip instead of two); each sum is formed in the same
// order as slot_sum forms it
__device__ __forceinline__ void slot_sum2(const Ctx& C, int sa, int sb, DF32& ra, DF32& rb) {
  const int l = threadIdx.x & 31;
  const float2* A = C.part + sa * kMaxPart;
  const float2* B = C.part + sb * kMaxPart;
  DF32 a{0.f, 0.f}, b{0.f, 0.f};
  for (int base = 0; base < C.nb; base += 32 * 8) {
    float2 va[8], vb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * 32 + l;
      va[u] = (i < C.nb) ? __ldcg(A + i) : make_float2(0.f, 0.f);
      vb[u] = (i < C.nb) ? __ldcg(B + i) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a = df_add(a, DF32{va[u].x, va[u].y});
      b = df_add(b, DF32{vb[u].x, vb[u].y});
    }
  }
  a = df_warp_sum(a);
  b = df_warp_sum(b);
  ra = DF32{__shfl_sync(0xffffffffu, a.hi, 0), __shfl_sync(0xffffffffu, a.lo, 0)};
  rb = DF32{__shfl_sync(0xffffffffu, b.hi, 0), __shfl_sync(0xffffffffu, b.lo, 0)};
}

// Convergence to the rounding floor: once gamma_k <= kCgrFloor gamma_0, the
// denominator delta_k - beta_k gamma_k / a_{k-1} is the difference of two
// rounding-level terms and may lose its sign; the CG then stops (a = 0 for the
// Newton step's remaining iterations) instead of reporting a breakdown.
constexpr double kCgrFloor = 1e-8;

// a_{k-1} and beta_{k-1} (k >= 1) from the partials of gamma_{k-1} (SLOT_RR0)
// and delta_{k-1} (SLOT_PQ) and the stored (gamma_{k-2}, a_{k-2}); every CTA
// derives the same values from the same partials, CTA 0 stores
// (gamma_{k-1}, a_{k-1}) for the next step (cgs[0..3] by parity of k), gamma_0
// (cgs[4]) and the stop flag (cgs[5]).  CTA-uniform; one block barrier.
__device__ __forceinline__ void cgr_scalars(const Ctx& C, int k, Scal2& a, Scal2& beta) {
  __shared__ Scal2 s_ab[2];
  if (threadIdx.x < 32) {
    DF32 gs, ds;
    slot_sum2(C, SLOT_RR0, SLOT_PQ, gs, ds);
    if (threadIdx.x == 0) {
      const double g = df_to_double(gs), d = df_to_double(ds);
      const double g0 = k == 1 ? g : C.cgs[4];
      bool stop = k > 1 && C.cgs[5] != 0.0;
      double bt = 0.0, den = d;
      if (k >= 2) {
        const double gp = C.cgs[2 * (k & 1)], ap = C.cgs[2 * (k & 1) + 1];
        bt = gp > 0.0 ? g / gp : 0.0;
        if (ap != 0.0) den = d - bt * g / ap;
      }
      double a64 = 0.0;
      if (!stop && g > 0.0) {
        if (den > 0.0 && isfinite(den)) {
          a64 = g / den;
        } else if (g <= kCgrFloor * g0) {
          stop = true;
        } else {
          raise_err(C, DEV_ENUMERIC);
        }
      }
      if (stop) bt = 0.0;
      if (C.bid == 0) {
        C.cgs[2 * ((k - 1) & 1)] = g;
        C.cgs[2 * ((k - 1) & 1) + 1] = a64;
        if (k == 1) C.cgs[4] = g;
        C.cgs[5] = stop ? 1.0 : 0.0;
      }
      const float ah = (float)a64, bh = (float)bt;
      s_ab[0] = Scal2{ah, (float)(a64 - (double)ah)};
      s_ab[1] = Scal2{bh, (float)(bt - (double)bh)};
    }
  }
  __syncthreads();
  a = s_ab[0];
  beta = s_ab[1];
}

// s_{k-1} and r_k of one element from r_{k-1}, w_{k-1}, s_{k-2} (k >= 2;
// s_0 = w_0): the one formula both the row items and the vector update use,
// so the items' on-the-fly residual is bit-identical to the stored one
__device__ __forceinline__ float2 cgr_s(float2 w, float2 s_old, Scal2 beta, bool rec) {
  return rec ? axpy2(s_old, beta, w) : w;
}
__device__ __forceinline__ float2 cgr_r(float2 r_old, float2 s, Scal2 na) { return axpy2(s, na, r_old); }

// ------------------------- R: the row pass of r_k and the step k-1 update
// Items (channel, TW rows): the row pass T(r_k) as phase_row_cg computes it,
// with r_k formed on the fly for k >= 1: its rho rows as cgr_r(r_{k-1},
// s_{k-1}) and its y-transformed coil part by linearity of H,
//   H s_{k-1} = H w_{k-1} + beta H s_{k-2},  H r_k = H r_{k-1} - a H s_{k-1},
// both written back in place (every element belongs to one thread of one
// item).  Every CTA first applies step k-1 to its share of the whole vector:
// p_{k-1}, s_{k-1}, x_k, r_k (new buffers; the old ones are only read, so the
// items may form their rows from them at the same time).
template <class K>
__device__ NLINV_PHASE void phase_row_cgr(const Ctx& C, float2* sm, int k) {
  constexpr int G1 = K::G1, G2 = K::G2, G = K::G, TW = K::TW, RS = K::RS;
  constexpr int EU = NLINV_EU;   // elements per thread per round of the vector update
  const int N = C.N, Gc = C.Gc, J = C.J;
  const int t = phase_tid();
  const bool upd = k > 0, rec = k > 1;
  const float2* r_old = C.rb[(k + 1) & 1];   // r_{k-1}
  float2* r_new = C.rb[k & 1];               // r_k (read when k == 0)
  const float2* w = C.q;                     // w_{k-1} = A r_{k-1}
  const float2* s_old = C.sb[k & 1];         // s_{k-2}
  float2* s_new = C.sb[(k + 1) & 1];         // s_{k-1}
  const float2* p_old = C.pb[k & 1];         // p_{k-2}
  float2* p_new = C.pb[(k + 1) & 1];         // p_{k-1}
  Scal2 a{0.f, 0.f}, beta{0.f, 0.f};
  // step k-1 on this CTA's share of the whole vector; the first round's loads
  // are issued before the scalars are fetched, so the two latencies overlap
  float2 rp[EU], wv[EU], so[EU], po[EU], xv[EU];
  const int stride = C.nb * blockDim.x;
  auto load = [&](int base) {
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const int e = base + t + u * stride;
      rp[u] = wv[u] = so[u] = po[u] = xv[u] = czero();
      if (e < C.nx) {
        rp[u] = ldcg(r_old + e);
        wv[u] = ldcg(w + e);
        if (rec) {
          so[u] = ldcg(s_old + e);
          po[u] = ldcg(p_old + e);
          xv[u] = ldcg(C.xcg + e);
        }
      }
    }
  };
  if (upd) load(C.bid * blockDim.x);
  if (upd) cgr_scalars(C, k, a, beta);
  const Scal2 na{-a.hi, -a.lo};
  if (upd) {
    for (int base = C.bid * blockDim.x; base < C.nx; base += EU * stride) {   // CTA-uniform
      if (base != C.bid * blockDim.x) load(base);
#pragma unroll
      for (int u = 0; u < EU; ++u) {
        const int e = base + t + u * stride;
        if (e < C.nx) {
          const float2 s = cgr_s(wv[u], so[u], beta, rec);
          const float2 p = rec ? axpy2(po[u], beta, rp[u]) : rp[u];
          s_new[e] = s;
          p_new[e] = p;
          C.xcg[e] = axpy2(p, a, xv[u]);
          r_new[e] = cgr_r(rp[u], s, na);
        }
      }
    }
  }
  const int groups = (N + TW - 1) / TW;
  const int items = J * groups;
  for (int it = C.bid; it < items; it += C.nb) {
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
        if (upd)
          rv[k1] = cgr_r(ldcg(r_old + ir), cgr_s(ldcg(w + ir), rec ? ldcg(s_old + ir) : czero(), beta, rec), na);
        else
          rv[k1] = ldcg(r_new + ir);
        cv[k1] = ldcg(C.c + (size_t)j * N * N + ir);
        rh[k1] = ldcg(C.xn + ir);
      }
    }
    {  // stage 1: thread (row, n1): H r_k of the band, inverse DFT over n2
      const int r1 = t / G1, n1 = t % G1, y1 = y0 + r1;
      if (r1 < TW && y1 < N) {
        float2 av[G2];
#pragma unroll
        for (int n2 = 0; n2 < G2; ++n2) {
          const int ix = coef_index(n1 + G1 * n2, G, Gc);
          av[n2] = czero();
          if (ix >= 0) {
            const size_t h = ((size_t)j * N + y1) * Gc + ix;
            if (upd) {
              const float2 hs = cgr_s(ldcg(C.Hw + h), rec ? ldcg(C.Hs + h) : czero(), beta, rec);
              const float2 hr = cgr_r(ldcg(C.Hr + h), hs, na);
              C.Hs[h] = hs;
              C.Hr[h] = hr;
              av[n2] = hr;
            } else {
              av[n2] = ldcg(C.Hr + h);
            }
          }
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
    {  // stage 3: thread (row, kb): forward DFT over k2 -> kb + G1 ka
      const int r3 = t / G1, kb = t % G1, y3 = y0 + r3;
      if (r3 < TW && y3 < N) {
        float2 d[G2];
#pragma unroll
        for (int a2 = 0; a2 < G2; ++a2) d[a2] = sm[r3 * RS + kb * (G2 + 1) + a2];
        dft<G2, false>(d);
        float2* dst = C.v + ((size_t)j * N + y3) * G;
#pragma unroll
        for (int ka = 0; ka < G2; ++ka) dst[kb + G1 * ka] = d[ka];
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------- F: the last step of the CG
// a_{K-1}, beta_{K-1}; p_{K-1} = r_{K-1} + beta p_{K-2};
// x^_{n+1} = x^_n + x_{K-1} + a p_{K-1}  (K >= 1)
template <class K>
__device__ __forceinline__ void phase_cgr_final(const Ctx& C, int Kcg) {
  constexpr int EU = NLINV_EU;
  const int t = threadIdx.x;
  const bool rec = Kcg > 1;
  const float2* r_last = C.rb[(Kcg + 1) & 1];   // r_{K-1}
  const float2* p_old = C.pb[Kcg & 1];          // p_{K-2}
  Scal2 a, beta;
  cgr_scalars(C, Kcg, a, beta);
  const int stride = C.nb * blockDim.x;
  for (int base = C.bid * blockDim.x; base < C.nx; base += EU * stride) {
    float2 rp[EU], po[EU], xv[EU], xo[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const int e = base + t + u * stride;
      rp[u] = po[u] = xv[u] = xo[u] = czero();
      if (e < C.nx) {
        rp[u] = ldcg(r_last + e);
        xo[u] = ldcg(C.xn + e);
        if (rec) {
          po[u] = ldcg(p_old + e);
          xv[u] = ldcg(C.xcg + e);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const int e = base + t + u * stride;
      if (e < C.nx) {
        const float2 p = rec ? axpy2(po[u], beta, rp[u]) : rp[u];
        C.xn[e] = cadd(xo[u], axpy2(p, a, xv[u]));
      }
    }
  }
}

}  // namespace nlinv
