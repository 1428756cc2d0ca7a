// Register-resident complex-FP32 DFT building blocks for the NLINV kernels.
//
// The paper (Sec. 2.2, Sec. 3.2) spends most of its time in batched 2-D FFTs
// on the twofold-oversampled grid.  Here a length-G transform is split as
// G = G1 * G2 ("four-step"): each thread holds one length-G2 (or G1) column
// of the G1 x G2 view entirely in registers, a compile-time mixed-radix DFT
// (radix 2/3/4/5/7, recursive Cooley-Tukey) transforms it, the inter-stage
// twiddle w_G^(n1 k2) is applied, and a single shared-memory exchange
// transposes the data for the second register DFT.  One 1-D transform thus
// costs one shared-memory round trip instead of one per radix stage.
//
// Twiddles of the in-register DFTs come from a __constant__ table holding
// exp(-2 pi i e / L) for every composite length L the recursion visits (one
// block of L entries per length), indexed by compile-time constants after
// unrolling, so they become constant-bank operands; the inter-stage twiddles
// w_G^e come from a per-grid table in global memory.  Both tables are
// computed on the host in double precision and rounded once to float.
#pragma once
#include <cuda_runtime.h>

namespace nlinv {

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cfma(float2 a, float s, float2 b) {  // a*s + b
  return make_float2(fmaf(a.x, s, b.x), fmaf(a.y, s, b.y));
}
__device__ __forceinline__ float2 czero() { return make_float2(0.f, 0.f); }

// multiply by -i (forward sign) or +i (inverse sign)
template <bool INV> __device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------- twiddle tables
// composite in-register DFT lengths (every length of the form 2^a 3^b 5^c 7^d
// that a compiled grid split reaches); block L of c_tw holds exp(-2 pi i e/L)
constexpr int kTwLens[] = {6, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 30, 32};
constexpr int kNumTwLens = sizeof(kTwLens) / sizeof(kTwLens[0]);
constexpr int tw_offset(int L) {
  int off = 0;
  for (int i = 0; i < kNumTwLens; ++i) {
    if (kTwLens[i] == L) return off;
    off += kTwLens[i];
  }
  return -1;
}
constexpr int tw_total() {
  int t = 0;
  for (int i = 0; i < kNumTwLens; ++i) t += kTwLens[i];
  return t;
}
constexpr int TWL = tw_total();            // entries of c_tw
__constant__ float2 c_tw[TWL];

constexpr float kSqrtHalf = 0.70710678118654752440f;

// a * w_L^e (w_L = exp(-2 pi i / L), conjugated for the inverse); e is a
// compile-time constant after unrolling, so the branches fold away.
template <int L, bool INV> __device__ __forceinline__ float2 twmul(float2 a, int e) {
  static_assert(tw_offset(L) >= 0, "in-register DFT length without a twiddle block (kTwLens)");
  e %= L;
  if (e == 0) return a;
  if (2 * e == L) return make_float2(-a.x, -a.y);
  if (4 * e == L) return mul_mi<INV>(a);
  if (4 * e == 3 * L) return mul_mi<!INV>(a);
  if (8 * e == L) {   // exp(-+ i pi/4)
    return INV ? make_float2((a.x - a.y) * kSqrtHalf, (a.x + a.y) * kSqrtHalf)
               : make_float2((a.x + a.y) * kSqrtHalf, (a.y - a.x) * kSqrtHalf);
  }
  if (8 * e == 3 * L) {  // exp(-+ 3 i pi/4)
    return INV ? make_float2((-a.x - a.y) * kSqrtHalf, (a.x - a.y) * kSqrtHalf)
               : make_float2((a.y - a.x) * kSqrtHalf, (-a.x - a.y) * kSqrtHalf);
  }
  float2 w = c_tw[tw_offset(L) + e];
  if (INV) w.y = -w.y;
  return cmul(a, w);
}

// ------------------------------------------------------- register DFTs
// In-place, natural order in and out: a[k] <- sum_n a[n] w_L^(nk).
template <int L> struct FirstFactor {
  static_assert(L % 2 == 0 || L % 3 == 0 || L % 5 == 0 || L % 7 == 0 || L == 1, "radix 2/3/4/5/7 only");
  static constexpr int value =
      (L % 4 == 0 && L != 4) ? 4 : (L % 2 == 0 ? 2 : (L % 3 == 0 ? 3 : (L % 5 == 0 ? 5 : 7)));
};

template <int L, bool INV> struct DFT {
  static __device__ __forceinline__ void run(float2 (&a)[L]) {
    // L = R * M: n = m + M r, k = k1 + R k2
    //   X[k1 + R k2] = sum_m w_M^(m k2) w_L^(m k1) sum_r a[m + M r] w_R^(r k1)
    constexpr int R = FirstFactor<L>::value;
    constexpr int M = L / R;
    static_assert(R * M == L, "bad factorisation");
    float2 t[L];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = a[m + M * r];
      DFT<R, INV>::run(v);
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) t[k1 * M + m] = twmul<L, INV>(v[k1], m * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      float2 u[M];
#pragma unroll
      for (int m = 0; m < M; ++m) u[m] = t[k1 * M + m];
      DFT<M, INV>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < M; ++k2) a[k1 + R * k2] = u[k2];
    }
  }
};

template <bool INV> struct DFT<1, INV> {
  static __device__ __forceinline__ void run(float2 (&)[1]) {}
};

template <bool INV> struct DFT<2, INV> {
  static __device__ __forceinline__ void run(float2 (&a)[2]) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};

template <bool INV> struct DFT<4, INV> {
  static __device__ __forceinline__ void run(float2 (&a)[4]) {
    float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    float2 t2 = cadd(a[1], a[3]), t3 = mul_mi<INV>(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};

// radix 3: w = exp(-+2 pi i/3) = -1/2 -+ i sqrt(3)/2
template <bool INV> struct DFT<3, INV> {
  static __device__ __forceinline__ void run(float2 (&a)[3]) {
    constexpr float s3 = 0.86602540378443864676f;   // sqrt(3)/2
    float2 t = cadd(a[1], a[2]);
    float2 d = mul_mi<INV>(cscale(csub(a[1], a[2]), s3));
    float2 m = cfma(t, -0.5f, a[0]);
    a[0] = cadd(a[0], t);
    a[1] = cadd(m, d);
    a[2] = csub(m, d);
  }
};

// radix 5 with cos/sin of 2 pi/5 and 4 pi/5 (closed forms in sqrt(5))
template <bool INV> struct DFT<5, INV> {
  static __device__ __forceinline__ void run(float2 (&a)[5]) {
    constexpr float c1 = 0.30901699437494742410f;   // (sqrt5 - 1)/4
    constexpr float c2 = -0.80901699437494742410f;  // -(sqrt5 + 1)/4
    constexpr float s1 = 0.95105651629515357212f;   // sqrt(10 + 2 sqrt5)/4
    constexpr float s2 = 0.58778525229247312917f;   // sqrt(10 - 2 sqrt5)/4
    float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
    float2 t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
    float2 m1 = cfma(t2, c2, cfma(t1, c1, a[0]));
    float2 m2 = cfma(t2, c1, cfma(t1, c2, a[0]));
    float2 n1 = cfma(t4, s2, cscale(t3, s1));
    float2 n2 = cfma(t4, -s1, cscale(t3, s2));
    n1 = mul_mi<INV>(n1);
    n2 = mul_mi<INV>(n2);
    a[0] = cadd(a[0], cadd(t1, t2));
    a[1] = cadd(m1, n1);
    a[4] = csub(m1, n1);
    a[2] = cadd(m2, n2);
    a[3] = csub(m2, n2);
  }
};

// radix 7: X_k = a0 + sum_m cos(2 pi m k/7) (a_m + a_{7-m})
//                   -+ i sum_m sin(2 pi m k/7) (a_m - a_{7-m}), m = 1..3,
// folding k and 7 - k; cos/sin of 2 pi m/7 as literals (m = 1, 2, 3)
template <bool INV> struct DFT<7, INV> {
  static __device__ __forceinline__ void run(float2 (&a)[7]) {
    constexpr float c1 = 0.62348980185873353053f, c2 = -0.22252093395631440429f, c3 = -0.90096886790241912624f;
    constexpr float s1 = 0.78183148246802980871f, s2 = 0.97492791218182360702f, s3 = 0.43388373911755812048f;
    const float2 t1 = cadd(a[1], a[6]), t2 = cadd(a[2], a[5]), t3 = cadd(a[3], a[4]);
    const float2 u1 = csub(a[1], a[6]), u2 = csub(a[2], a[5]), u3 = csub(a[3], a[4]);
    const float2 m1 = cfma(t3, c3, cfma(t2, c2, cfma(t1, c1, a[0])));
    const float2 m2 = cfma(t3, c1, cfma(t2, c3, cfma(t1, c2, a[0])));
    const float2 m3 = cfma(t3, c2, cfma(t2, c1, cfma(t1, c3, a[0])));
    // sin(2 pi m k / 7) for k = 1, 2, 3: (s1 s2 s3), (s2 -s3 -s1), (s3 -s1 s2)
    const float2 n1 = mul_mi<INV>(cfma(u3, s3, cfma(u2, s2, cscale(u1, s1))));
    const float2 n2 = mul_mi<INV>(cfma(u3, -s1, cfma(u2, -s3, cscale(u1, s2))));
    const float2 n3 = mul_mi<INV>(cfma(u3, s2, cfma(u2, -s1, cscale(u1, s3))));
    a[0] = cadd(a[0], cadd(t1, cadd(t2, t3)));
    a[1] = cadd(m1, n1);
    a[6] = csub(m1, n1);
    a[2] = cadd(m2, n2);
    a[5] = csub(m2, n2);
    a[3] = cadd(m3, n3);
    a[4] = csub(m3, n3);
  }
};

template <int L, bool INV> __device__ __forceinline__ void dft(float2 (&a)[L]) { DFT<L, INV>::run(a); }

// inter-stage twiddle w_G^e from the per-grid table (e < G); conj for INV
template <bool INV> __device__ __forceinline__ float2 twg(const float2* __restrict__ tw, int e) {
  float2 w = __ldg(tw + e);
  if (INV) w.y = -w.y;
  return w;
}

}  // namespace nlinv
