// C-ABI implementation of the GB300 NLINV hot path (see include/nlinv.h).
//
// The host side: argument checks, plans, the batch and stream schedulers and
// the reverse-mode driver.  The kernels of the hot path live in grid.cuh,
// compiled once per FFT grid size (grid.cu) and reached through the GridOps
// table of each size; the preprocessing kernels (PSF of a trajectory,
// gridding by the adjoint NDFT) and the reverse mode's vector kernels are
// here.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.h"

using namespace nlinv;

namespace nlinv {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? NLINV_ENOMEM : NLINV_ECUDA;
}

const GridOps* grid_ops(int G, int N) {
#define NLINV_PICK_OPS(a, b, n, tw, mb) \
  if (G == (a) * (b) && N == (n) && grid_ops_##a##_##b##_##n) return grid_ops_##a##_##b##_##n();
  NLINV_GRIDS(NLINV_PICK_OPS)
#undef NLINV_PICK_OPS
  return nullptr;
}

}  // namespace nlinv

namespace {

// ------------------------------------------------ temporal median filter
// out[i] = median over the window of |img_t[i]| (T odd, T <= kMaxMedian):
// one thread per pixel, the T magnitudes sorted in registers (insertion
// sort over compile-time-bounded loops)
constexpr int kMaxMedian = 15;
struct MedianWindow {
  const float2* img[kMaxMedian];
};
__global__ void k_median(int T, long long n, MedianWindow W, float* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float v[kMaxMedian];
#pragma unroll
    for (int t = 0; t < kMaxMedian; ++t) {
      if (t < T) {
        const float2 z = W.img[t][i];
        v[t] = sqrtf(z.x * z.x + z.y * z.y);
      }
    }
#pragma unroll
    for (int a = 1; a < kMaxMedian; ++a) {
      if (a < T) {
#pragma unroll
        for (int b = a; b > 0; --b) {
          const float lo = fminf(v[b - 1], v[b]), hi = fmaxf(v[b - 1], v[b]);
          v[b - 1] = lo;
          v[b] = hi;
        }
      }
    }
    float m = v[0];
#pragma unroll
    for (int t = 0; t < kMaxMedian; ++t)
      if (t == T / 2) m = v[t];
    out[i] = m;
  }
}

// ------------------------------------------- convolution gridding (NUFFT)
// Kaiser-Bessel gridding of the preprocessing stage (Sec. 3.1): kernel
// phi(u) = I0(beta sqrt(1 - (2u/W)^2)) on W grid points, modulated by the
// centre c = N/2 of the field of view; continuous transform
// Phi(t) = W sinh(s)/s, s = sqrt(beta^2 - (pi W t)^2).
constexpr int kMaxKbWidth = 16;

double kb_beta(int W, double sigma) {
  return M_PI * std::sqrt((W / sigma) * (W / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
}

// per sample and axis: the first grid point f0 of the W nearest to p = G k
// and the W complex weights phi(f - p) exp(-2 pi i (f - p) c / G) (FP64)
__global__ void k_kb_weights(int S, int G, int W, double beta, double c, const double* __restrict__ kxy, float2* w,
                             int* f0) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
#pragma unroll 1
  for (int ax = 0; ax < 2; ++ax) {
    const double p = G * kxy[2 * s + ax];
    const int f = (int)floor(p - 0.5 * W) + 1;
    f0[2 * s + ax] = f;
    for (int i = 0; i < W; ++i) {
      const double u = f + i - p;
      const double a = 1.0 - (2.0 * u / W) * (2.0 * u / W);
      const double ph = a >= 0.0 ? cyl_bessel_i0(beta * sqrt(a)) : 0.0;
      double sn, cs;
      sincospi(-2.0 * u * c / G, &sn, &cs);
      w[((size_t)s * 2 + ax) * W + i] = make_float2((float)(ph * cs), (float)(ph * sn));
    }
  }
}

// dap[i] = 1 / Phi((i - N/2) / G)  (FP64)
__global__ void k_kb_deapod(int N, int G, int W, double beta, float* dap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double t = (i - 0.5 * N) / G;
  const double sarg = sqrt(beta * beta - (M_PI * W * t) * (M_PI * W * t));
  dap[i] = (float)(sarg / (W * sinh(sarg)));
}

// Z[j][fy][fx] += y[j][s] wy wx over the W x W points of sample s (periodic);
// one thread per (sample, channel), float2 atomics in global memory
__global__ void k_kb_spread(int S, int J, int G, int W, const float2* __restrict__ y, const float2* __restrict__ w,
                            const int* __restrict__ f0, float2* Z) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= (long long)S * J) return;
  const int s = (int)(id % S), j = (int)(id / S);
  const float2 yv = y[(size_t)j * S + s];
  const float2* wx = w + (size_t)s * 2 * W;
  const float2* wy = wx + W;
  const int fx0 = f0[2 * s], fy0 = f0[2 * s + 1];
  float2* Zj = Z + (size_t)j * G * G;
  for (int a = 0; a < W; ++a) {
    const int fy = ((fy0 + a) % G + G) % G;
    const float2 ya = cmul(yv, wy[a]);
    for (int b = 0; b < W; ++b) {
      const int fx = ((fx0 + b) % G + G) % G;
      atomicAdd(Zj + (size_t)fy * G + fx, cmul(ya, wx[b]));
    }
  }
}

bool supported_grid(int G, int N) { return grid_ops(G, N) != nullptr; }

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

int check_plan(const nlinv_plan_s* pl) { return pl ? NLINV_OK : NLINV_EINVAL; }

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

int nlinv_grid_list(int* G_out, int* N_out, int cap) {
  int n = 0;
#define NLINV_LIST_GRID(a, b, nr, tw, mb)           \
  if (grid_ops_##a##_##b##_##nr) {                  \
    if (n < cap && G_out) G_out[n] = (a) * (b);     \
    if (n < cap && N_out) N_out[n] = (nr);          \
    ++n;                                            \
  }
  NLINV_GRIDS(NLINV_LIST_GRID)
#undef NLINV_LIST_GRID
  return n;
}

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
  p->G = 0;
  p->cluster_cs = 0;
  return NLINV_OK;
}

int nlinv_plan(nlinv_plan_t* out, const nlinv_params_t* p, const float* psf, nlinv_stream_t stream) {
  if (!out || !p) return NLINV_EINVAL;
  *out = nullptr;
  const int N = p->N, G = p->G ? p->G : 2 * p->N, J = p->J;
  const int Gc = p->Gc ? p->Gc : G / 4;
  if (N <= 0 || J <= 0 || J > 4096) return NLINV_EINVAL;
  if (G < 2 * N) return NLINV_EINVAL;
  if (!supported_grid(G, N)) return NLINV_EUNSUPPORTED;
  if (Gc < 2 || Gc > G) return NLINV_EINVAL;
  if (p->newton_steps < 1 || p->newton_steps > kMaxNewton) return NLINV_EINVAL;
  if (p->cg_iters < 0 || p->cg_iters > 4096) return NLINV_EINVAL;
  if (p->n_turns < 1 || p->n_turns > 1024) return NLINV_EINVAL;
  if (!(p->alpha0 > 0.0) || !(p->q > 0.0) || p->q > 1.0 || !(p->damping >= 0.0)) return NLINV_EINVAL;
  if (!(p->w_a >= 0.0) || !(p->w_l >= 0.0)) return NLINV_EINVAL;
  if (p->exec_mode < 0 || p->exec_mode > 4) return NLINV_EINVAL;
  if (p->max_batch < 0 || p->max_batch > kMaxBatch) return NLINV_EINVAL;
  if (p->cluster_cs < 0 || p->cluster_cs > 16) return NLINV_EINVAL;
  if (psf && ((uintptr_t)psf & 3u)) return NLINV_EINVAL;

  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const GridOps* ops = grid_ops(G, N);

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
  take(nx * f2);                         // 21 s_0 (A p of the per-phase CG)
  take(nx * f2);                         // 22 s_1
  take((size_t)J * N * Gc * f2);         // 23 Hw
  take((size_t)J * N * Gc * f2);         // 24 Hs
  take(6 * sizeof(double));              // 25 cgs
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
  C.sb[0] = (float2*)(base + off[21]);
  C.sb[1] = (float2*)(base + off[22]);
  C.Hw = (float2*)(base + off[23]);
  C.Hs = (float2*)(base + off[24]);
  C.cgs = (double*)(base + off[25]);
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

  rc = ops->setup(pl);
  if (rc == NLINV_OK) {
    if ((e = cudaStreamCreateWithFlags(&pl->aux, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&pl->ev_done, cudaEventDisableTiming)) != cudaSuccess)
      rc = cuda_fail(e, "plan streams");
  }
  if (rc != NLINV_OK) return fail(rc);
  *out = pl;
  return NLINV_OK;
}

int nlinv_plan_destroy(nlinv_plan_t pl) {
  if (!pl) return NLINV_EINVAL;
  for (auto& g : pl->vjp_graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    cudaFree(g.stage);
  }
  cudaFree(pl->vjp_mem);
  for (cudaStream_t s2 : pl->vjp_st) cudaStreamDestroy(s2);
  for (cudaEvent_t e2 : pl->vjp_ev) cudaEventDestroy(e2);
  if (pl->vjp_fork) cudaEventDestroy(pl->vjp_fork);
  if (pl->vjp_host) cudaFreeHost(pl->vjp_host);
  for (auto& g : pl->pgraphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (pl->gcap) cudaStreamDestroy(pl->gcap);
  cudaFree(pl->io_dev);
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

int nlinv_plan_path(nlinv_plan_t pl, int* exec_path, int* cluster_size) {
  RC(check_plan(pl));
  const int m = pl->prm.exec_mode;
  const int path = m == 0 ? 4 : ((m == 1 || m == 4) ? m : (m == 3 && pl->cl_cs > 0 ? 3 : 2));
  if (exec_path) *exec_path = path;
  if (cluster_size) *cluster_size = path == 3 ? pl->cl_cs : 0;
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
                                                                         1.0 / (4.0 * pl->N * pl->N));
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
      N, S, (const float2*)y, Ex, Ey, pl->C.s, (float)(0.5 / pl->N));
  CKL("k_adj_ndft");
  return grid_ops(pl->G, pl->N)->grid_fwd(pl, st, (float2*)Y_out);
}

int nlinv_grid_nufft(nlinv_plan_t pl, int S, const double* kxy, const void* y, int W, void* Y_out,
                     nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (S <= 0 || !kxy || !y || !Y_out || ((uintptr_t)kxy & 7u) || !aligned8(y) || !aligned8(Y_out))
    return NLINV_EINVAL;
  if (W < 2 || W > kMaxKbWidth) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int N = pl->N, G = pl->G, J = pl->J;
  const size_t zb = align_up((size_t)J * G * G * sizeof(float2));
  const size_t wb = align_up((size_t)S * 2 * W * sizeof(float2));
  const size_t bb = align_up((size_t)S * 2 * sizeof(int));
  RC(ensure_prep(pl, zb + wb + bb + align_up((size_t)N * sizeof(float))));
  char* base = (char*)pl->prep;
  float2* Z = (float2*)base;
  float2* w = (float2*)(base + zb);
  int* f0 = (int*)(base + zb + wb);
  float* dap = (float*)(base + zb + wb + bb);
  const double beta = kb_beta(W, (double)G / N);
  CK(cudaMemsetAsync(Z, 0, (size_t)J * G * G * sizeof(float2), st));
  k_kb_weights<<<(S + 127) / 128, 128, 0, st>>>(S, G, W, beta, 0.5 * N, kxy, w, f0);
  CKL("k_kb_weights");
  k_kb_deapod<<<(N + 127) / 128, 128, 0, st>>>(N, G, W, beta, dap);
  CKL("k_kb_deapod");
  const long long nt = (long long)S * J;
  k_kb_spread<<<(int)((nt + 255) / 256), 256, 0, st>>>(S, J, G, W, (const float2*)y, w, f0, Z);
  CKL("k_kb_spread");
  return grid_ops(pl->G, pl->N)->grid_kb(pl, st, Z, dap, (float)((double)G / (2.0 * N)), (float2*)Y_out);
}

int nlinv_median(const void* const* imgs, int T, long long n, float* out, nlinv_stream_t stream) {
  if (!imgs || !out || n <= 0 || T < 1 || T > kMaxMedian || (T % 2) == 0 || ((uintptr_t)out & 3u))
    return NLINV_EINVAL;
  MedianWindow W;
  std::memset(&W, 0, sizeof(W));
  for (int t = 0; t < T; ++t) {
    if (!imgs[t] || !aligned8(imgs[t])) return NLINV_EINVAL;
    W.img[t] = (const float2*)imgs[t];
  }
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  k_median<<<(int)g, 256, 0, (cudaStream_t)stream>>>(T, n, W, out);
  CKL("k_median");
  return NLINV_OK;
}

int nlinv_apply_DF(nlinv_plan_t pl, const void* xhat, const void* dx, void* z, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!xhat || !dx || !z || !aligned8(xhat) || !aligned8(dx) || !aligned8(z)) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  return grid_ops(pl->G, pl->N)->DF(pl, st, (const float2*)xhat, (const float2*)dx, (float2*)z, false);
}

int nlinv_apply_DFH(nlinv_plan_t pl, const void* xhat, const void* z, void* dx_out, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!xhat || !z || !dx_out || !aligned8(xhat) || !aligned8(z) || !aligned8(dx_out)) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  return grid_ops(pl->G, pl->N)->DFH(pl, st, (const float2*)xhat, (const float2*)z, (float2*)dx_out, false);
}

int nlinv_apply_normal(nlinv_plan_t pl, const void* xhat, const void* dx, int turn, double alpha, void* out,
                       nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!xhat || !dx || !out || !aligned8(xhat) || !aligned8(dx) || !aligned8(out)) return NLINV_EINVAL;
  if (turn < 0 || turn >= pl->U || !(alpha >= 0.0)) return NLINV_EINVAL;
  if (out == xhat || out == dx) return NLINV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const float* P = pl->psf + (size_t)turn * pl->G * pl->G;
  return grid_ops(pl->G, pl->N)->normal(pl, st, (const float2*)xhat, (const float2*)dx, P, alpha, (float2*)out, false);
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
  return grid_ops(pl->G, pl->N)->frame(pl, st, F);
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
    const int rc = grid_ops(pl->G, pl->N)->batch(pl, gs, B, grid);
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
  RC(grid_ops(G, G / 2)->prepare());
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
  if (!supported_grid(G, N)) return NLINV_EUNSUPPORTED;
  if (Gc == 0) Gc = G / 4;
  if (Gc < 2 || Gc > G) return NLINV_EINVAL;
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

  // a plan view of the static array: the per-size operations read the sizes
  // from the plan and the buffers from its Ctx
  nlinv_plan_s tmp;
  tmp.N = N;
  tmp.G = G;
  tmp.Gc = Gc;
  tmp.J = J;
  tmp.U = 1;
  tmp.nx = (long long)N * N + (long long)J * Gc * Gc;
  tmp.psf = const_cast<float*>(psf);
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
  return grid_ops(G, N)->normal(&tmp, st, (const float2*)xhat, (const float2*)dx, psf, alpha, (float2*)out, false);
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
// A forward sweep records every Newton step: the checkpoint x^_n, the
// residual z and the whole CG tape (p_k, q_k, r_k; 3 K + 1 vectors per step,
// ~0.24 GB per frame at N = 160 with 10 channels), and the reverse sweep
// reverses each CG step by step from that record.  All scalars (the CG tape
// and the adjoint scalars) are computed and kept on the device in FP64, so a
// frame's reverse pass is issued without host synchronisation and frames of
// a batch run on their own streams.
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

// y = s x + b y with s = mul * (*sp), a device FP64 scalar applied as a float pair
__global__ void k_axpby_s(long long n, float2* y, const float2* x, const double* sp, double mul, float b) {
  const double sv = mul * *sp;
  const float hi = (float)sv, lo = (float)(sv - (double)hi);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 xv = x[i];
    float2 base = make_float2(0.f, 0.f);
    if (b != 0.f) {
      const float2 yv = y[i];
      base = make_float2(b * yv.x, b * yv.y);
    }
    y[i] = make_float2(fmaf(hi, xv.x, fmaf(lo, xv.x, base.x)), fmaf(hi, xv.y, fmaf(lo, xv.y, base.y)));
  }
}

// Device scalars of one frame's reverse pass (FP64), offsets into one array:
// the CG tape of the Newton step being reversed (rho_k = |r_k|^2, a_k,
// beta_k, gamma_k = Re<p_k, A p_k>, act_k = 1 for a step CG executed), the
// adjoint scalars rhobar_k, the eight inner products D of a reverse step,
// the coefficients of its vector updates, and alpha-bar / alpha0-bar.
struct VjpSlots {
  int rho, a, beta, gamma, act, rhobar, D, co, ab, a0b, t1, t2, c0, err, total;
  explicit VjpSlots(int K) {
    int o = 0;
    auto take = [&](int n) {
      const int r = o;
      o += n;
      return r;
    };
    rho = take(K + 1);
    a = take(K > 0 ? K : 1);
    beta = take(K > 0 ? K : 1);
    gamma = take(K > 0 ? K : 1);
    act = take(K > 0 ? K : 1);
    rhobar = take(K + 1);
    D = take(kMaxDots);
    co = take(8);
    ab = take(1);
    a0b = take(1);
    t1 = take(1);
    t2 = take(1);
    c0 = take(1);
    err = take(1);
    total = o;
  }
};

// float pair (hi, lo) of an FP64 coefficient: hi + lo carries it to ~2^-48
struct Coef {
  float hi, lo;
  __device__ explicit Coef(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  // c * x + y, in the rounding order of k_axpby / k_axpby_s with b = 1
  __device__ float2 fma2(float2 x, float2 y) const {
    return make_float2(fmaf(hi, x.x, fmaf(lo, x.x, y.x)), fmaf(hi, x.y, fmaf(lo, x.y, y.y)));
  }
  // c * x (b = 0)
  __device__ float2 mul2(float2 x) const {
    return make_float2(fmaf(hi, x.x, fmaf(lo, x.x, 0.f)), fmaf(hi, x.y, fmaf(lo, x.y, 0.f)));
  }
};

// block sum of an FP64 partial into part[blockIdx.x]
__device__ __forceinline__ void block_partial(double acc, double* part) {
  __shared__ double sw[32];
  acc = warp_sum_f64(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sw[w];
    part[blockIdx.x] = a;
  }
}

// CG step k of the recorded forward sweep in one pass: a_k = rho_k / gamma_k
// for an executed step (rho_k > 0; a breakdown gamma_k <= 0 flags an error
// and stops), else 0 -- every block derives it, block 0 records it --, then
// x += a_k p_k, r_{k+1} = r_k - a_k q_k and the per-block FP64 partials of
// |r_{k+1}|^2.  Launched with kDotBlocks x 256 threads, so the partials are
// those k_dot_part forms over r_{k+1}.
__global__ void k_cg_step(long long n, double* sc, VjpSlots S, int k, float2* xcg, const float2* __restrict__ p,
                          const float2* __restrict__ q, const float2* r, float2* r1, double* part) {
  const double rho = sc[S.rho + k], g = sc[S.gamma + k];
  double act = rho > 0.0 ? 1.0 : 0.0;
  const bool broke = act != 0.0 && !(g > 0.0 && isfinite(g));
  if (broke) act = 0.0;
  const double a = act != 0.0 ? rho / g : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (broke) sc[S.err] = 1.0;
    sc[S.act + k] = act;
    sc[S.a + k] = a;
  }
  const Coef ca(a), cn(-a);
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    xcg[i] = ca.fma2(p[i], xcg[i]);
    const float2 rv = cn.fma2(q[i], r[i]);
    r1[i] = rv;
    acc = fma((double)rv.x, (double)rv.x, fma((double)rv.y, (double)rv.y, acc));
  }
  block_partial(acc, part);
}

// beta_k = rho_{k+1} / rho_k for an executed step, else 0 (block 0 records
// it) and, when p1 is given, the next direction p_{k+1} = r_{k+1} + beta_k p_k
__global__ void k_cg_dir(long long n, double* sc, VjpSlots S, int k, float2* p1, const float2* __restrict__ r1,
                         const float2* __restrict__ p) {
  const double beta = sc[S.act + k] != 0.0 ? sc[S.rho + k + 1] / sc[S.rho + k] : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[S.beta + k] = beta;
  if (!p1) return;
  const Coef cb(beta);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p1[i] = cb.fma2(p[i], r1[i]);
}

// Reverse of CG step k from its inner products D (see nlinv_frame_vjp):
// the adjoint scalars and the coefficients of the step's vector updates
//   co0: rbar += co0 pbar   co1: pb = co1 pbar   co2: rbar += co2 r_{k+1}
//   co3: qbar = co3 rbar    co4: pb += co4 xb    co5: pb += co5 q, qbar += co5 p
// For a step CG did not execute every update is the identity.
__global__ void k_rev_step(double* sc, VjpSlots S, int k) {
  double* co = sc + S.co;
  if (sc[S.act + k] == 0.0) {
    co[0] = 0.0;
    co[1] = 1.0;
    co[2] = co[3] = co[4] = co[5] = 0.0;
    return;
  }
  const double* D = sc + S.D;
  const double a = sc[S.a + k], beta = sc[S.beta + k], gamma = sc[S.gamma + k];
  const double rk = sc[S.rho + k], rk1 = sc[S.rho + k + 1];
  double* rhobar = sc + S.rhobar;
  const double betabar = D[0];                     // p_{k+1} = r_{k+1} + beta p_k
  rhobar[k + 1] += betabar / rk;                   // beta = rho_{k+1} / rho_k
  rhobar[k] -= betabar * rk1 / (rk * rk);
  const double c = 2.0 * rhobar[k + 1];            // rho_{k+1} = <r, r>
  const double abar = -(D[1] + D[2] + c * D[3]) + D[4];   // r -= a q; x += a p
  rhobar[k] += abar / gamma;                       // a = rho_k / gamma_k
  const double gammabar = -abar * rk / (gamma * gamma);
  sc[S.ab] += -a * (D[5] + D[0] + c * D[6]) + gammabar * D[7];
  co[0] = 1.0;
  co[1] = beta;
  co[2] = c;
  co[3] = -a;
  co[4] = a;
  co[5] = gammabar;
}

// the vector updates of reverse CG step k with the coefficients co of
// k_rev_step, in the order (and rounding) of seven k_axpby_s passes:
//   rbar += co0 pbar;  pb = co1 pbar;  rbar += co2 r1;  qbar = co3 rbar;
//   pb += co4 xb;  pb += co5 q;  qbar += co5 p
__global__ void k_rev_update(long long n, const double* __restrict__ co, float2* rbar, const float2* __restrict__ pbar,
                             float2* pb, const float2* __restrict__ r1, float2* qbar, const float2* __restrict__ xb,
                             const float2* __restrict__ q, const float2* __restrict__ p) {
  const Coef c0(co[0]), c1(co[1]), c2(co[2]), c3(co[3]), c4(co[4]), c5(co[5]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 pv = pbar[i];
    float2 rv = c0.fma2(pv, rbar[i]);
    float2 bv = c1.mul2(pv);
    rv = c2.fma2(r1[i], rv);
    float2 qv = c3.mul2(rv);
    bv = c4.fma2(xb[i], bv);
    bv = c5.fma2(q[i], bv);
    qv = c5.fma2(p[i], qv);
    rbar[i] = rv;
    pb[i] = bv;
    qbar[i] = qv;
  }
}

// pb += t0;  xbn = (xbn + t1) + t2  (three k_axpby passes with a = b = 1)
__global__ void k_rev_acc(long long n, float2* pb, const float2* __restrict__ t0, float2* xbn,
                          const float2* __restrict__ t1, const float2* __restrict__ t2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 a = pb[i], b = t0[i];
    pb[i] = make_float2(a.x + b.x, a.y + b.y);
    const float2 x = xbn[i], u = t1[i], v = t2[i];
    xbn[i] = make_float2((x.x + u.x) + v.x, (x.y + u.y) + v.y);
  }
}

// end of a reverse Newton step: 2 rhobar_0 (p_0 = r_0 = b) ...
__global__ void k_rev_c0(double* sc, VjpSlots S) { sc[S.c0] = 2.0 * sc[S.rhobar]; }
// ... and alpha-bar -= <bbar, x - x_ref>, alpha0-bar += q^n alpha-bar
__global__ void k_rev_alpha(double* sc, VjpSlots S, double qn) {
  sc[S.ab] -= sc[S.t1] - sc[S.t2];
  sc[S.a0b] += qn * sc[S.ab];
}

__global__ void k_fill(double* p, int n, double v) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = v;
}

// Each Newton step n of a frame keeps its scalars in its own block of
// S.total doubles.  out[f] = alpha0-bar of frame f, the sum of the blocks'
// a0b in the order the reverse sweep reaches them (n = M-1 .. 0);
// out[nf + f] = 1 if any block flagged a breakdown.
__global__ void k_gather_vjp(int nf, int M, const double* sc0, size_t stride, VjpSlots S, double* out) {
  const int f = threadIdx.x;
  if (f < nf) {
    const double* sc = sc0 + f * stride;
    double a = 0.0, e = 0.0;
    for (int n = M - 1; n >= 0; --n) {
      a += sc[(size_t)n * S.total + S.a0b];
      if (sc[(size_t)n * S.total + S.err] != 0.0) e = 1.0;
    }
    out[f] = a;
    out[nf + f] = e;
  }
}

// z <- s P z on [J][G][G]
__global__ void k_psf_scale(int J, int G, float2* z, const float* __restrict__ P, float s) {
  const long long n = (long long)J * G * G, g2 = (long long)G * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = cscale(z[i], s * P[i % g2]);
}

// z1 <- s P z1, z2 <- s P z2 on [J][G][G]
__global__ void k_psf_scale2(int J, int G, float2* z1, float2* z2, const float* __restrict__ P, float s) {
  const long long n = (long long)J * G * G, g2 = (long long)G * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float pk = s * P[i % g2];
    z1[i] = cscale(z1[i], pk);
    z2[i] = cscale(z2[i], pk);
  }
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
  const nlinv_plan_s* pl;   // the plan, or a view of it on one frame workspace
  cudaStream_t st;
  const float* P;
  long long nx, nk;
  double* part;   // [kMaxDots][kDotBlocks]
  const GridOps* ops;
  // The plan's coil-map buffer holds W^-1 of lin's coil part when
  // coils_at == lin.  lin is the Newton step's checkpoint x^_n, which is not
  // written while it is the linearisation point; maps of any other point
  // (a buffer that may change between calls) are never reused.  With `alt`
  // (a view whose coil-map buffer is a scratch array) the maps of other
  // points go there, so lin's maps survive them.
  const nlinv_plan_s* alt = nullptr;
  const float2* lin = nullptr;
  mutable const float2* coils_at = nullptr;
  // the view whose coil buffer serves point w
  const nlinv_plan_s* at(const float2* w) const { return (w != nullptr && w == lin) || !alt ? pl : alt; }
  // whether that coil buffer already holds the maps of w; updates the record
  bool coils_ready(const float2* w) const {
    if (w != nullptr && w == lin) {
      const bool ready = coils_at == lin;
      coils_at = lin;
      return ready;
    }
    if (!alt) coils_at = nullptr;   // the plan's buffer is about to hold another point's maps
    return false;
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
  // Re<u, v> into the device scalar *out (FP64; nothing is read back)
  int dot(const float2* u, const float2* v, long long n, double* out) const {
    k_dot_part<<<kDotBlocks, 256, 0, st>>>(n, u, v, part);
    CKL("k_dot_part");
    k_dot_final<<<1, 32, 0, st>>>(kDotBlocks, part, out);
    CKL("k_dot_final");
    return NLINV_OK;
  }
  // kMaxDots products Re<u_j, v_j> into the device scalars out[0..kMaxDots)
  int dots(const DotSet& S, double* out) const {
    k_dots_part<kMaxDots><<<kDotBlocks, 256, 0, st>>>(nx, S, part);
    CKL("k_dots_part");
    k_dots_final<<<kMaxDots, 32, 0, st>>>(kDotBlocks, part, out);
    CKL("k_dots_final");
    return NLINV_OK;
  }
  // y = (mul * *s) x + b y with the device scalar s
  int axpby_s(float2* y, const float2* x, const double* s, double mul, double b, long long n) const {
    k_axpby_s<<<grid(n), 256, 0, st>>>(n, y, x, s, mul, (float)b);
    CKL("k_axpby_s");
    return NLINV_OK;
  }
  // z = DF(x)[d]
  int DF(const float2* x, const float2* d, float2* z) const {
    const bool r = coils_ready(x);
    return ops->DF(at(x), st, x, d, z, r);
  }
  // out = DF(w)^H z
  int DFH(const float2* w, const float2* z, float2* out) const {
    const bool r = coils_ready(w);
    return ops->DFH(at(w), st, w, z, out, r);
  }
  // out = (DF(x)^H P DF(x) + alpha) d
  int normal(const float2* x, const float2* d, double alpha, float2* out) const {
    const bool r = coils_ready(x);
    return ops->normal(at(x), st, x, d, P, alpha, out, r);
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

// One frame's reverse-pass workspace.  The forward sweep keeps, for every
// Newton step n, its CG tape (p_k, q_k, r_k), its residual z = Y - P F(x^_n)
// and its block of device scalars; at(n) points tp / tq / tr / z / sc at
// step n's copies.  The other vectors are shared by the steps.
struct GradWS {
  float2 *ck, *b, *z, *zt, *zt2, *tp, *tq, *tr, *xb, *xbn, *pbar, *rbar, *qbar, *pb, *t0, *t1, *t2, *xref,
      *xrefbar, *xcg;
  float2* cscr;   // coil maps [J][N][N] of points other than the linearisation point
  double *part, *sc;
  size_t vn = 0;                             // elements of one vector slot (256-byte aligned)
  size_t spq = 0, sr = 0, sz = 0, ssc = 0;   // elements between two Newton steps' tapes / z / scalars
  GradWS at(int n) const {
    GradWS u = *this;
    u.tp += (size_t)n * spq;
    u.tq += (size_t)n * spq;
    u.tr += (size_t)n * sr;
    u.z += (size_t)n * sz;
    u.sc += (size_t)n * ssc;
    return u;
  }
};

// bytes of one frame's reverse-pass workspace (a multiple of 256): M + 1
// checkpoints, M tapes of 2 kt + Kc + 1 vectors, 13 shared vectors, M + 2
// k-space arrays, the dot partials and M scalar blocks
size_t grad_ws_bytes(const nlinv_plan_s* pl) {
  const int M = pl->prm.newton_steps, Kc = pl->prm.cg_iters;
  const size_t nx = (size_t)pl->nx, nk = (size_t)pl->J * pl->G * pl->G;
  const size_t vb = align_up(nx * sizeof(float2)), kb = align_up(nk * sizeof(float2));
  const size_t kt = Kc > 0 ? Kc : 1;   // p_k and q_k tapes (one vector even without CG)
  return vb * ((M + 1) + (size_t)M * (2 * kt + Kc + 1) + 13) + (M + 2) * kb +
         align_up((size_t)pl->J * pl->N * pl->N * sizeof(float2)) +
         align_up((size_t)kMaxDots * kDotBlocks * sizeof(double)) +
         align_up((size_t)M * VjpSlots(Kc).total * sizeof(double));
}

void grad_ws_carve(const nlinv_plan_s* pl, char* p, GradWS& w) {
  const int M = pl->prm.newton_steps, Kc = pl->prm.cg_iters;
  const size_t nx = (size_t)pl->nx, nk = (size_t)pl->J * pl->G * pl->G;
  const size_t vb = align_up(nx * sizeof(float2)), kb = align_up(nk * sizeof(float2));
  const size_t kt = Kc > 0 ? Kc : 1;
  auto vec = [&](size_t count) {
    float2* r = (float2*)p;
    p += vb * count;
    return r;
  };
  w.ck = vec(M + 1);
  w.tp = vec(M * kt);
  w.tq = vec(M * kt);
  w.tr = vec((size_t)M * (Kc + 1));
  w.b = vec(1);
  w.xb = vec(1);
  w.xbn = vec(1);
  w.pbar = vec(1);
  w.rbar = vec(1);
  w.qbar = vec(1);
  w.pb = vec(1);
  w.t0 = vec(1);
  w.t1 = vec(1);
  w.t2 = vec(1);
  w.xref = vec(1);
  w.xrefbar = vec(1);
  w.xcg = vec(1);
  w.z = (float2*)p;
  p += kb * M;
  w.zt = (float2*)p;
  p += kb;
  w.zt2 = (float2*)p;
  p += kb;
  w.cscr = (float2*)p;
  p += align_up((size_t)pl->J * pl->N * pl->N * sizeof(float2));
  w.part = (double*)p;
  p += align_up((size_t)kMaxDots * kDotBlocks * sizeof(double));
  w.sc = (double*)p;
  w.vn = vb / sizeof(float2);
  w.spq = kt * w.vn;
  w.sr = (size_t)(Kc + 1) * w.vn;
  w.sz = kb / sizeof(float2);
  w.ssc = (size_t)VjpSlots(Kc).total;
}

// b = DF(x)^H (Y - P F^(x)) - alpha (x - xref); leaves the residual in w.z
int grad_rhs(const GradOps& O, const GradWS& w, const float2* Y, const float2* x, double alpha, float2* b) {
  RC(O.DF(x, x, w.z));
  RC(O.resid(w.z, Y));
  RC(O.DFH(x, w.z, b));
  RC(O.axpby(b, x, -alpha, 1.0, O.nx));
  return O.axpby(b, w.xref, alpha, 1.0, O.nx);
}

// CG from zero recording p_k, q_k, r_k and the tape scalars (device) in w's
// Newton-step copies; the step delta in w.xcg.  Every one of the `iters`
// steps is issued: a step after an exactly zero residual has a_k = beta_k = 0
// and leaves the vectors unchanged (the host cannot see the residual without
// a read-back).  Per step: q = A p, <p, q>, one pass for a_k, x, r_{k+1} and
// the partials of |r_{k+1}|^2, their sum, one pass for beta_k and p_{k+1}.
int grad_cg(const GradOps& O, const GradWS& w, const VjpSlots& S, const float2* x, double alpha, const float2* b,
            int iters) {
  const long long nx = O.nx;
  double* sc = w.sc;
  float2* r0 = w.tr;
  RC(O.copy(r0, b, nx));
  RC(O.zero(w.xcg, nx));
  RC(O.dot(r0, r0, nx, sc + S.rho));
  if (iters > 0) RC(O.copy(w.tp, r0, nx));
  for (int k = 0; k < iters; ++k) {
    float2* p = w.tp + (size_t)k * w.vn;
    float2* q = w.tq + (size_t)k * w.vn;
    float2* r = w.tr + (size_t)k * w.vn;
    float2* r1 = w.tr + (size_t)(k + 1) * w.vn;
    RC(O.normal(x, p, alpha, q));
    RC(O.dot(p, q, nx, sc + S.gamma + k));
    k_cg_step<<<kDotBlocks, 256, 0, O.st>>>(nx, sc, S, k, w.xcg, p, q, r, r1, O.part);
    CKL("k_cg_step");
    k_dot_final<<<1, 32, 0, O.st>>>(kDotBlocks, O.part, sc + S.rho + k + 1);
    CKL("k_dot_final");
    float2* p1 = k + 1 < iters ? w.tp + (size_t)(k + 1) * w.vn : nullptr;
    k_cg_dir<<<p1 ? O.grid(nx) : 1, 256, 0, O.st>>>(p1 ? nx : 0, sc, S, k, p1, r1, p);
    CKL("k_cg_dir");
  }
  return NLINV_OK;
}

// The whole reverse pass of one frame, issued on `st` without any host
// synchronisation; alpha0-bar and the breakdown flags end up in the Newton
// steps' scalar blocks (k_gather_vjp).  The forward sweep records every
// Newton step's CG (the workspace holds all M tapes), so the reverse sweep
// reads them instead of recomputing the step from its checkpoint.
int vjp_issue(const nlinv_plan_s* view, cudaStream_t st, const GradWS& w, const float* P, const float2* Yd,
              const float2* xprev, const float2* gbar, float2* Ybar, float2* xprev_bar) {
  const nlinv_params_t& prm = view->prm;
  const int M = prm.newton_steps, Kc = prm.cg_iters;
  const VjpSlots S(Kc);
  GradOps O{view, st, P, view->nx, (long long)view->J * view->G * view->G, w.part, grid_ops(view->G, view->N)};
  // coil maps of points other than x^_n (the reverse steps' DF^H at q-bar,
  // p and b-bar) go to a scratch array, so x^_n's maps are built once per
  // Newton step
  nlinv_plan_s alt(*view);
  alt.C.c = w.cscr;
  O.alt = &alt;
  const long long nx = O.nx, nk = O.nk;
  const int nfill = M * S.total;
  k_fill<<<(nfill + 255) / 256, 256, 0, st>>>(w.sc, nfill, 0.0);
  CKL("k_fill");
  // x^_0 and x_ref
  if (xprev) {
    RC(O.copy(w.ck, xprev, nx));
  } else {
    k_init_x<<<O.grid(nx), 256, 0, st>>>((int)nx, view->N * view->N, w.ck);
    CKL("k_init_x");
  }
  RC(O.copy(w.xref, w.ck, nx));
  RC(O.axpby(w.xref, w.xref, 0.0, prm.damping, nx));
  // forward: checkpoints x^_n, each Newton step's residual and CG tape
  for (int n = 0; n < M; ++n) {
    const GradWS u = w.at(n);
    const float2* x = w.ck + (size_t)n * w.vn;
    float2* x1 = w.ck + (size_t)(n + 1) * w.vn;
    const double alpha = prm.alpha0 * std::pow(prm.q, n);
    O.lin = x;
    RC(grad_rhs(O, u, Yd, x, alpha, w.b));
    RC(grad_cg(O, u, S, x, alpha, w.b, Kc));
    RC(O.copy(x1, x, nx));
    RC(O.axpby(x1, w.xcg, 1.0, 1.0, nx));
  }
  // reverse
  RC(O.zero(Ybar, nk));
  RC(O.zero(w.xrefbar, nx));
  RC(O.copy(w.xb, gbar, nx));
  GradWS v = w;   // xb / xbn swap roles per Newton step as host pointers
  for (int n = M - 1; n >= 0; --n) {
    GradWS u = v.at(n);   // step n's tape, residual and scalars; pbar / pb swap per CG step
    double* sc = u.sc;
    const float2* x = w.ck + (size_t)n * w.vn;
    const double alpha = prm.alpha0 * std::pow(prm.q, n);
    O.lin = x;
    RC(O.copy(u.xbn, u.xb, nx));                      // x^_{n+1} = x^_n + delta
    RC(O.zero(u.pbar, nx));
    RC(O.zero(u.rbar, nx));
    for (int k = Kc - 1; k >= 0; --k) {
      const float2* p = u.tp + (size_t)k * w.vn;
      const float2* q = u.tq + (size_t)k * w.vn;
      const float2* r1 = u.tr + (size_t)(k + 1) * w.vn;
      // every inner product this step needs, from the vectors as they enter
      // it (the updates below are linear in them):
      //   D0 <p, pbar>  D1 <q, rbar>  D2 <q, pbar>  D3 <q, r1>
      //   D4 <p, xb>    D5 <p, rbar>  D6 <p, r1>    D7 <p, p>
      DotSet DS;
      const float2* U[kMaxDots] = {p, q, q, q, p, p, p, p};
      const float2* V[kMaxDots] = {u.pbar, u.rbar, u.pbar, r1, u.xb, u.rbar, r1, p};
      for (int j = 0; j < kMaxDots; ++j) {
        DS.u[j] = U[j];
        DS.v[j] = V[j];
      }
      RC(O.dots(DS, sc + S.D));
      k_rev_step<<<1, 1, 0, st>>>(sc, S, k);          // adjoint scalars, coefficients co
      CKL("k_rev_step");
      // p_{k+1} = r_{k+1} + beta p_k;  rho_{k+1} = <r, r>;  r_{k+1} = r_k - a q_k;
      // x_{k+1} = x_k + a p_k;  gamma = <p, q>
      k_rev_update<<<O.grid(nx), 256, 0, st>>>(nx, sc + S.co, u.rbar, u.pbar, u.pb, r1, u.qbar, u.xb, q, p);
      CKL("k_rev_update");
      RC(O.normal(x, u.qbar, alpha, u.t0));                  // q = A p
      // A depends on x^_n: both DF at x^_n first, while its coil maps are current
      RC(O.DF(x, p, u.zt));
      RC(O.DF(x, u.qbar, u.zt2));
      k_psf_scale2<<<O.grid(nk), 256, 0, st>>>(view->J, view->G, u.zt, u.zt2, P, 1.f);
      CKL("k_psf_scale2");
      RC(O.DFH(u.qbar, u.zt, u.t1));
      RC(O.DFH(p, u.zt2, u.t2));
      k_rev_acc<<<O.grid(nx), 256, 0, st>>>(nx, u.pb, u.t0, u.xbn, u.t1, u.t2);
      CKL("k_rev_acc");
      std::swap(u.pbar, u.pb);
    }
    // p_0 = r_0 = b, rho_0 = <r_0, r_0>:  b-bar
    RC(O.axpby(u.rbar, u.pbar, 1.0, 1.0, nx));
    k_rev_c0<<<1, 1, 0, st>>>(sc, S);
    CKL("k_rev_c0");
    RC(O.axpby_s(u.rbar, u.tr, sc + S.c0, 1.0, 1.0, nx));
    const float2* bbar = u.rbar;
    // right-hand side
    RC(O.DFH(bbar, u.z, u.t1));
    RC(O.axpby(u.xbn, u.t1, 1.0, 1.0, nx));
    RC(O.DF(x, bbar, u.zt));
    k_axpby<<<O.grid(nk), 256, 0, st>>>(nk, Ybar, u.zt, 1.f, 0.f, 1.f);   // Y-bar += DF(x) b-bar
    CKL("k_axpby");
    RC(O.psf(u.zt, 1.f));
    RC(O.DFH(x, u.zt, u.t1));
    RC(O.axpby(u.xbn, u.t1, -1.0, 1.0, nx));
    RC(O.axpby(u.xbn, bbar, -alpha, 1.0, nx));
    RC(O.dot(bbar, x, nx, sc + S.t1));
    RC(O.dot(bbar, w.xref, nx, sc + S.t2));
    k_rev_alpha<<<1, 1, 0, st>>>(sc, S, std::pow(prm.q, n));
    CKL("k_rev_alpha");
    RC(O.axpby(w.xrefbar, bbar, alpha, 1.0, nx));
    v.xb = u.xbn;
    v.xbn = u.xb;
    v.pbar = u.pbar;
    v.pb = u.pb;
  }
  if (xprev_bar) {
    if (xprev) {
      RC(O.copy(xprev_bar, v.xb, nx));
      RC(O.axpby(xprev_bar, w.xrefbar, prm.damping, 1.0, nx));
    } else {
      RC(O.zero(xprev_bar, nx));
    }
  }
  return NLINV_OK;
}

}  // namespace

extern "C" int nlinv_set_alpha0(nlinv_plan_t pl, double alpha0) {
  if (!pl || !(alpha0 > 0.0)) return NLINV_EINVAL;
  pl->prm.alpha0 = alpha0;
  return NLINV_OK;
}

extern "C" int nlinv_batch_vjp(nlinv_plan_t pl, int nframes, const void* const* Y, const int* turns,
                               const void* const* x_prev, const void* const* gbar, void* const* Ybar_out,
                               double* alpha0_bar_out, void* const* xprev_bar_out, nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (nframes <= 0 || nframes > pl->max_batch || !Y || !turns || !gbar || !Ybar_out) return NLINV_EINVAL;
  for (int f = 0; f < nframes; ++f) {
    if (!Y[f] || !gbar[f] || !Ybar_out[f] || !aligned8(Y[f]) || !aligned8(gbar[f]) || !aligned8(Ybar_out[f]))
      return NLINV_EINVAL;
    if ((x_prev && x_prev[f] && !aligned8(x_prev[f])) || (xprev_bar_out && xprev_bar_out[f] && !aligned8(xprev_bar_out[f])))
      return NLINV_EINVAL;
    if (turns[f] < 0 || turns[f] >= pl->U) return NLINV_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t wsb = grad_ws_bytes(pl);
  const size_t need = wsb * nframes + align_up(2 * kMaxBatch * sizeof(double));
  if (pl->vjp_bytes < need) {   // a new workspace: every captured reverse pass is stale
    for (auto& g : pl->vjp_graphs)
      if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
      }
    if (pl->vjp_mem) CK(cudaFree(pl->vjp_mem));
    pl->vjp_mem = nullptr;
    pl->vjp_bytes = 0;
    CK(cudaMalloc(&pl->vjp_mem, need));
    pl->vjp_bytes = need;
  }
  char* wbase = (char*)pl->vjp_mem;
  double* gather = (double*)(wbase + wsb * nframes);
  if (!pl->vjp_host) CK(cudaMallocHost(&pl->vjp_host, 2 * kMaxBatch * sizeof(double)));
  if (!pl->vjp_fork) CK(cudaEventCreateWithFlags(&pl->vjp_fork, cudaEventDisableTiming));
  while ((int)pl->vjp_st.size() < nframes) {
    cudaStream_t s2 = nullptr;
    cudaEvent_t e2 = nullptr;
    CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    pl->vjp_st.push_back(s2);
    CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    pl->vjp_ev.push_back(e2);
    pl->vjp_graphs.emplace_back();
  }
  const size_t nx = (size_t)pl->nx, nk = (size_t)pl->J * pl->G * pl->G;
  const size_t sy = align_up(nk * sizeof(float2)), sx = align_up(nx * sizeof(float2));
  CK(cudaEventRecord(pl->vjp_fork, st));
  // each frame on its own stream, workspace and reverse-pass slot: the slot's
  // reverse pass is captured once into a CUDA graph (no host synchronisation
  // inside it) reading and writing the slot's staging buffers, and replayed
  for (int f = 0; f < nframes; ++f) {
    nlinv_plan_s::VjpGraph& vg = pl->vjp_graphs[f];
    if (!vg.stage) CK(cudaMalloc(&vg.stage, 2 * sy + 3 * sx));
    float2* sY = (float2*)vg.stage;
    float2* sYbar = (float2*)((char*)vg.stage + sy);
    float2* sg = (float2*)((char*)vg.stage + 2 * sy);
    float2* sxp = (float2*)((char*)vg.stage + 2 * sy + sx);
    float2* sxpb = (float2*)((char*)vg.stage + 2 * sy + 2 * sx);
    const int has_xp = (x_prev && x_prev[f]) ? 1 : 0;
    const int want_xpb = (xprev_bar_out && xprev_bar_out[f]) ? 1 : 0;
    cudaStream_t sf = pl->vjp_st[f];
    if (!vg.exec || vg.alpha0 != pl->prm.alpha0 || vg.turn != turns[f] || vg.has_xprev != has_xp ||
        vg.want_xprev_bar != want_xpb) {
      if (vg.exec) {
        cudaGraphExecDestroy(vg.exec);
        vg.exec = nullptr;
      }
      nlinv_plan_s view(*pl);
      view.C = frame_ctx(pl->C, (size_t)f * pl->fstride);
      // frames' reverse passes run side by side: each operator launch takes
      // its share of two waves of resident CTAs (one CTA per item when alone;
      // 8 frames: C5 backward 60.4 -> 55.9 ms)
      view.op_grid = nframes > 1 ? (2 * pl->op_minb * pl->nsm + nframes - 1) / nframes : 0;
      GradWS w;
      grad_ws_carve(pl, wbase + wsb * f, w);
      CK(cudaStreamBeginCapture(sf, cudaStreamCaptureModeThreadLocal));
      const int rc = vjp_issue(&view, sf, w, pl->psf + (size_t)turns[f] * pl->G * pl->G, sY,
                               has_xp ? sxp : nullptr, sg, sYbar, want_xpb ? sxpb : nullptr);
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(sf, &graph);
      if (rc != NLINV_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      CK(ec);
      const cudaError_t ei = cudaGraphInstantiate(&vg.exec, graph, 0);
      cudaGraphDestroy(graph);
      CK(ei);
      vg.alpha0 = pl->prm.alpha0;
      vg.turn = turns[f];
      vg.has_xprev = has_xp;
      vg.want_xprev_bar = want_xpb;
    }
    CK(cudaStreamWaitEvent(sf, pl->vjp_fork, 0));
    CK(cudaMemcpyAsync(sY, Y[f], nk * sizeof(float2), cudaMemcpyDeviceToDevice, sf));
    CK(cudaMemcpyAsync(sg, gbar[f], nx * sizeof(float2), cudaMemcpyDeviceToDevice, sf));
    if (has_xp) CK(cudaMemcpyAsync(sxp, x_prev[f], nx * sizeof(float2), cudaMemcpyDeviceToDevice, sf));
    CK(cudaGraphLaunch(vg.exec, sf));
    CK(cudaMemcpyAsync(Ybar_out[f], sYbar, nk * sizeof(float2), cudaMemcpyDeviceToDevice, sf));
    if (want_xpb) CK(cudaMemcpyAsync(xprev_bar_out[f], sxpb, nx * sizeof(float2), cudaMemcpyDeviceToDevice, sf));
    CK(cudaEventRecord(pl->vjp_ev[f], sf));
    CK(cudaStreamWaitEvent(st, pl->vjp_ev[f], 0));
  }
  GradWS w0;
  grad_ws_carve(pl, wbase, w0);
  k_gather_vjp<<<1, 64, 0, st>>>(nframes, pl->prm.newton_steps, w0.sc, wsb / sizeof(double),
                                 VjpSlots(pl->prm.cg_iters), gather);
  CKL("k_gather_vjp");
  CK(cudaMemcpyAsync(pl->vjp_host, gather, 2 * nframes * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int f = 0; f < nframes; ++f)
    if (pl->vjp_host[nframes + f] != 0.0) return NLINV_ENUMERIC;
  if (alpha0_bar_out)
    for (int f = 0; f < nframes; ++f) alpha0_bar_out[f] = pl->vjp_host[f];
  return NLINV_OK;
}

extern "C" int nlinv_frame_vjp(nlinv_plan_t pl, const void* Y, int turn, const void* x_prev, const void* gbar,
                               void* Ybar_out, double* alpha0_bar_out, void* xprev_bar_out,
                               nlinv_stream_t stream) {
  RC(check_plan(pl));
  if (!Y || !gbar || !Ybar_out) return NLINV_EINVAL;
  const void* xp = x_prev;
  void* xb = xprev_bar_out;
  return nlinv_batch_vjp(pl, 1, &Y, &turn, &xp, &gbar, &Ybar_out, alpha0_bar_out, &xb, stream);
}

#ifdef NLINV_TIMELINE
// profiling builds: the timeline and stage sums of grid size G's unit
extern "C" int nlinv_debug_timeline(int G, int N, unsigned long long* host, int n) {
  const GridOps* o = grid_ops(G, N);
  return o ? o->timeline(host, n) : NLINV_EUNSUPPORTED;
}
extern "C" int nlinv_debug_stages(int G, int N, unsigned long long* ns, unsigned long long* cnt) {
  const GridOps* o = grid_ops(G, N);
  return o ? o->stages(ns, cnt) : NLINV_EUNSUPPORTED;
}
#endif
