// CG / Chebyshev vector kernels and the solve drivers.
//
// Krylov scalars live on the device (SolveState); every reduction is a
// two-stage deterministic sum (per-CTA partials, then the last CTA to
// finish adds them in CTA order and updates the scalars), accumulated in
// FP64 whatever the vector precision.  Every kernel of an iteration returns
// immediately once the state says "done", so the host can queue a chunk of
// iterations (captured once as a CUDA graph) and only read the status word
// between chunks.
//
// Algorithms (readings of the paper: CG with a Jacobi or Chebyshev-Jacobi
// preconditioner, Sec. 3.5 / Sec. 6.1; single-precision inner solver with
// double-precision correction, Sec. 6.1):
//   PCG: x0 = 0, r = b, z = P r, p = z; alpha = (r,z)/(p,Kp); x += alpha p;
//        r -= alpha Kp; stop when ||r||_2 <= tol ||b||_2; beta = (r+,z+)/(r,z);
//        p = z+ + beta p.
//   Chebyshev(m) on [lo, hi] for D^-1 K: theta = (hi+lo)/2, delta = (hi-lo)/2,
//        sigma = theta/delta, rho_0 = 1/sigma; d = D^-1 r / theta, z = d;
//        for i = 1..m-1: rho_i = 1/(2 sigma - rho_{i-1});
//        d = rho_i rho_{i-1} d + 2 rho_i / delta D^-1 (r - K z); z += d.
//   lambda_max: largest eigenvalue of the Lanczos tridiagonal built from
//        the first CG coefficients (T_ii = 1/a_i + b_{i-1}/a_{i-1},
//        T_i,i+1 = sqrt(b_i)/a_i), by Sturm-sequence bisection.
//   Mixed: x = 0; repeat r = b - K64 x (FP64), stop if ||r|| <= tol ||b||;
//        solve K32 d = r/||r|| to inner_tol with FP32 PCG; x += ||r|| d.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "mfx_internal.h"

namespace mfx {

constexpr int kRedThreads = 256;
constexpr int kMaxRedBlocks = 1024;
constexpr int kMaxLanczos = 128;

struct SolveState {
  double rz, pq, rr, bb, tol2, alpha, beta, pad0;
  int32_t done, status, it, max_it;
  int32_t record, pad1, pad2, pad3;
  double lan_alpha[kMaxLanczos], lan_beta[kMaxLanczos];
};

int reduction_blocks(int64_t n) {
  const int64_t b = (n + kRedThreads * 4 - 1) / (kRedThreads * 4);
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, std::min(kMaxRedBlocks, device_sm_count() * 4)));
}

// Block sum of NV values; thread 0 gets the totals.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kRedThreads / 32];
#pragma unroll
  for (int j = 0; j < NV; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[j][warp] = v[j];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      v[j] = lane < kRedThreads / 32 ? sh[j][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    }
  }
}

// The (p, q), update and rz kernels of CG take four strides of the grid per step with all their loads
// issued first (one stride per step held too few loads in flight: 1.5-2 TB/s), and add the step's four
// products in the vectors' precision before one FP64 accumulation (GB300's FP64 rate is 1/64 of FP32).
constexpr int kSteps = 4;

template <typename Real>
__device__ __forceinline__ void load_steps(const Real* __restrict__ a, int64_t i, int64_t S, Real (&v)[kSteps]) {
#pragma unroll
  for (int u = 0; u < kSteps; ++u) v[u] = a[i + u * S];
}

template <typename Real>
__device__ __forceinline__ double dot_steps(const Real (&a)[kSteps], const Real (&b)[kSteps]) {
  Real t = a[0] * b[0];
#pragma unroll
  for (int u = 1; u < kSteps; ++u) t += a[u] * b[u];
  return (double)t;
}

// Writes the CTA partials; returns true in the last CTA, whose thread 0 then holds the totals.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, unsigned int* counter) {
  block_sum<NV>(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) partials[blockIdx.x * NV + j] = v[j];
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // the last CTA sums the partials: strided loads from L2 by all its threads, then a block sum (one
  // thread walking them in turn waits on hundreds of dependent round trips: 40-80 us at 600 CTAs)
  double t[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) t[j] = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int j = 0; j < NV; ++j) t[j] += __ldcg(partials + b * NV + j);
  block_sum<NV>(t);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = t[j];
    *counter = 0u;
  }
  return true;
}

template <typename Real>
__global__ void dot_kernel(int64_t n, const Real* __restrict__ a, const Real* __restrict__ b, double* result,
                           double* partials, unsigned int* counter) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += (double)a[i] * (double)b[i];
  if (grid_sum<1>(v, partials, counter) && threadIdx.x == 0) *result = v[0];
}

// PCG start: x = 0, r = b, bb = (b,b); with Jacobi also rz = (r, D^-1 r) and p = D^-1 r.
template <typename Real>
__global__ void cg_init_kernel(int64_t n, const Real* __restrict__ b, Real* __restrict__ x, Real* __restrict__ r,
                               Real* __restrict__ p, const Real* __restrict__ dinv, bool jacobi, SolveState* st,
                               double* partials, unsigned int* counter) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Real bi = b[i];
    x[i] = Real(0);
    r[i] = bi;
    v[0] += (double)bi * (double)bi;
    if (jacobi) {
      const Real z = dinv[i] * bi;
      p[i] = z;
      v[1] += (double)bi * (double)z;
    }
  }
  if (grid_sum<2>(v, partials, counter) && threadIdx.x == 0) {
    st->bb = v[0];
    st->rr = v[0];
    st->rz = v[1];
    st->it = 0;
    st->status = MFX_OK;
    st->done = (v[0] == 0.0) ? 1 : 0;
    if (!isfinite(v[0])) {
      st->done = 1;
      st->status = MFX_BREAKDOWN;
    }
  }
}

// pq = (p, q); alpha = rz / pq.
template <typename Real>
__global__ void cg_pq_kernel(int64_t n, const Real* __restrict__ p, const Real* __restrict__ q, SolveState* st,
                             double* partials, unsigned int* counter) {
  if (st->done) return;
  double v[1] = {0.0};
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kSteps - 1) * S < n; i += kSteps * S) {
    Real a[kSteps], b[kSteps];
    load_steps(p, i, S, a);
    load_steps(q, i, S, b);
    v[0] += dot_steps(a, b);
  }
  for (; i < n; i += S) v[0] += (double)p[i] * (double)q[i];
  if (grid_sum<1>(v, partials, counter) && threadIdx.x == 0) {
    st->pq = v[0];
    if (!(v[0] > 0.0) || !isfinite(v[0])) {
      st->status = MFX_BREAKDOWN;
      st->done = 1;
    } else {
      st->alpha = st->rz / v[0];
      if (st->record && st->it < kMaxLanczos) st->lan_alpha[st->it] = st->alpha;
    }
  }
}

// x += alpha p; r -= alpha q; rr = (r, r); with Jacobi also rz+ = (r, D^-1 r) and beta.
template <typename Real>
__global__ void cg_update_kernel(int64_t n, Real* __restrict__ x, Real* __restrict__ r, const Real* __restrict__ p,
                                 const Real* __restrict__ q, const Real* __restrict__ dinv, bool jacobi,
                                 SolveState* st, double* partials, unsigned int* counter) {
  if (st->done) return;
  const Real alpha = (Real)st->alpha;
  double v[2] = {0.0, 0.0};
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kSteps - 1) * S < n; i += kSteps * S) {
    Real xv[kSteps], pv[kSteps], rv[kSteps], qv[kSteps], dv[kSteps];
    load_steps(x, i, S, xv);
    load_steps(p, i, S, pv);
    load_steps(r, i, S, rv);
    load_steps(q, i, S, qv);
    if (jacobi) load_steps(dinv, i, S, dv);
#pragma unroll
    for (int u = 0; u < kSteps; ++u) {
      x[i + u * S] = xv[u] + alpha * pv[u];
      rv[u] = rv[u] - alpha * qv[u];
      r[i + u * S] = rv[u];
      if (jacobi) dv[u] *= rv[u];
    }
    v[0] += dot_steps(rv, rv);
    if (jacobi) v[1] += dot_steps(rv, dv);
  }
  for (; i < n; i += S) {
    x[i] += alpha * p[i];
    const Real ri = r[i] - alpha * q[i];
    r[i] = ri;
    v[0] += (double)ri * (double)ri;
    if (jacobi) v[1] += (double)ri * (double)(dinv[i] * ri);
  }
  if (grid_sum<2>(v, partials, counter) && threadIdx.x == 0) {
    st->rr = v[0];
    st->it += 1;
    if (!isfinite(v[0])) {
      st->status = MFX_BREAKDOWN;
      st->done = 1;
    } else if (v[0] <= st->tol2 * st->bb) {
      st->status = MFX_OK;
      st->done = 1;
    } else if (st->it >= st->max_it) {
      st->status = MFX_NOT_CONVERGED;
      st->done = 1;
    }
    if (jacobi) {
      st->beta = v[1] / st->rz;
      st->rz = v[1];
      if (st->record && st->it - 1 < kMaxLanczos) st->lan_beta[st->it - 1] = st->beta;
    }
  }
}

// rz+ = (r, z); beta = rz+ / rz (Chebyshev-preconditioned CG).
template <typename Real>
__global__ void cg_rz_kernel(int64_t n, const Real* __restrict__ r, const Real* __restrict__ z, SolveState* st,
                             double* partials, unsigned int* counter) {
  if (st->done) return;
  double v[1] = {0.0};
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kSteps - 1) * S < n; i += kSteps * S) {
    Real a[kSteps], b[kSteps];
    load_steps(r, i, S, a);
    load_steps(z, i, S, b);
    v[0] += dot_steps(a, b);
  }
  for (; i < n; i += S) v[0] += (double)r[i] * (double)z[i];
  if (grid_sum<1>(v, partials, counter) && threadIdx.x == 0) {
    st->beta = v[0] / st->rz;
    st->rz = v[0];
  }
}

// p = z + beta p, with z = D^-1 r (jacobi) or z given.
template <typename Real>
__global__ void cg_p_kernel(int64_t n, Real* __restrict__ p, const Real* __restrict__ r,
                            const Real* __restrict__ dinv, const Real* __restrict__ z, const SolveState* st) {
  if (st->done) return;
  const Real beta = (Real)st->beta;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kSteps - 1) * S < n; i += kSteps * S) {
    Real pv[kSteps], a[kSteps], b[kSteps];
    load_steps(p, i, S, pv);
    if (z) {
      load_steps(z, i, S, a);
    } else {
      load_steps(dinv, i, S, a);
      load_steps(r, i, S, b);
#pragma unroll
      for (int u = 0; u < kSteps; ++u) a[u] *= b[u];
    }
#pragma unroll
    for (int u = 0; u < kSteps; ++u) p[i + u * S] = a[u] + beta * pv[u];
  }
  for (; i < n; i += S) {
    const Real zi = z ? z[i] : dinv[i] * r[i];
    p[i] = zi + beta * p[i];
  }
}

// Chebyshev start: d = D^-1 r / theta, z = d.
template <typename Real>
__global__ void cheb_init_kernel(int64_t n, const Real* __restrict__ r, const Real* __restrict__ dinv,
                                 Real* __restrict__ d, Real* __restrict__ z, Real inv_theta, const int32_t* skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Real v = dinv[i] * r[i] * inv_theta;
    d[i] = v;
    z[i] = v;
  }
}

// Chebyshev step: d = c1 d + c2 D^-1 (r - Kz); z += d.
template <typename Real>
__global__ void cheb_step_kernel(int64_t n, const Real* __restrict__ r, const Real* __restrict__ kz,
                                 const Real* __restrict__ dinv, Real* __restrict__ d, Real* __restrict__ z, Real c1,
                                 Real c2, const int32_t* skip) {
  if (skip && *skip) return;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kSteps - 1) * S < n; i += kSteps * S) {
    Real dv[kSteps], iv[kSteps], rv[kSteps], kv[kSteps], zv[kSteps];
    load_steps(d, i, S, dv);
    load_steps(dinv, i, S, iv);
    load_steps(r, i, S, rv);
    load_steps(kz, i, S, kv);
    load_steps(z, i, S, zv);
#pragma unroll
    for (int u = 0; u < kSteps; ++u) {
      const Real di = c1 * dv[u] + c2 * iv[u] * (rv[u] - kv[u]);
      d[i + u * S] = di;
      z[i + u * S] = zv[u] + di;
    }
  }
  for (; i < n; i += S) {
    const Real di = c1 * d[i] + c2 * dinv[i] * (r[i] - kz[i]);
    d[i] = di;
    z[i] += di;
  }
}

template <typename Real>
__global__ void reciprocal_kernel(int64_t n, const Real* __restrict__ d, Real* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = Real(1) / d[i];
}

// r64 = b - y; out: (r, r)
__global__ void residual_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ y,
                                double* __restrict__ r, double* result, double* partials, unsigned int* counter) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - y[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  if (grid_sum<1>(v, partials, counter) && threadIdx.x == 0) *result = v[0];
}

__global__ void scale_to_f32_kernel(int64_t n, const double* __restrict__ r, const double* scale_sq,
                                    float* __restrict__ out) {
  const double s = 1.0 / sqrt(*scale_sq);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)(r[i] * s);
}

__global__ void add_scaled_f32_kernel(int64_t n, double* __restrict__ x, const float* __restrict__ d,
                                      const double* scale_sq) {
  const double s = sqrt(*scale_sq);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += s * (double)d[i];
}

template <typename Real>
__global__ void convert_kernel(int64_t n, const double* __restrict__ in, Real* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (Real)in[i];
}

// ------------------------------------------------------------------ host side

static int vec_grid(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)device_sm_count() * 8));
}

mfx_status launch_dot(const mfx_op* op, mfx_prec prec, int64_t n, const void* a, const void* b, double* result,
                      cudaStream_t s) {
  const int g = reduction_blocks(n);
  if (prec == MFX_F64)
    dot_kernel<double><<<g, kRedThreads, 0, s>>>(n, (const double*)a, (const double*)b, result, op->d_partials,
                                                  op->d_counter);
  else
    dot_kernel<float><<<g, kRedThreads, 0, s>>>(n, (const float*)a, (const float*)b, result, op->d_partials,
                                                 op->d_counter);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

// Workspace of one precision.
template <typename Real>
struct Work {
  Real *x, *r, *p, *q, *z, *d, *t, *dinv, *b;
};

struct SolveWorkspace {
  size_t bytes = 0;
  void* base = nullptr;
  SolveState* st = nullptr;
  double* scal = nullptr;  // misc FP64 device scalars
  Work<double> w64{};
  Work<float> w32{};
  double* r64 = nullptr;   // mixed: FP64 residual
  double* y64 = nullptr;   // mixed: K64 x
  SolveState* h_st = nullptr;  // pinned host copy
  double lambda_max[2] = {0.0, 0.0};
  cudaStream_t stream = nullptr;  // solver stream (graph capture needs a non-default stream)
};

static SolveWorkspace* workspace(mfx_op* op) { return reinterpret_cast<SolveWorkspace*>(op->d_work); }

// Pinned host blocks for the solver status words, cut from slabs that live as long as the process:
// taking and returning a block needs no CUDA call (cudaFreeHost would synchronise the device).
static constexpr size_t kPinBlock = (sizeof(SolveState) + 255) / 256 * 256;
static std::mutex g_pin_lock;
static std::vector<void*> g_pin_free;

static SolveState* pinned_status_get() {
  std::lock_guard<std::mutex> g(g_pin_lock);
  if (g_pin_free.empty()) {
    constexpr int kPerSlab = 32;
    void* slab = nullptr;
    if (cudaMallocHost(&slab, kPinBlock * kPerSlab) != cudaSuccess) return nullptr;
    for (int i = kPerSlab - 1; i >= 0; --i) g_pin_free.push_back((char*)slab + i * kPinBlock);
  }
  void* p = g_pin_free.back();
  g_pin_free.pop_back();
  return (SolveState*)p;
}

static void pinned_status_put(SolveState* p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_pin_lock);
  g_pin_free.push_back(p);
}

// Solver workspace: one stream-ordered device allocation (no device-wide synchronisation when it
// is made or freed), a pinned status block and a stream of its own.
static mfx_status ensure_workspace(mfx_op* op) {
  if (op->d_work) return MFX_OK;
  auto* ws = new (std::nothrow) SolveWorkspace();
  if (!ws) return set_error(MFX_ENOMEM, "solver workspace: host allocation failed");
  const int64_t n = op->n_dofs;
  const size_t n64 = (size_t)n * sizeof(double), n32 = (size_t)n * sizeof(float);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t total = al(sizeof(SolveState)) + al(64 * sizeof(double));
  if (op->has_f64) total += 9 * al(n64);
  if (op->has_f32) total += 9 * al(n32) + 2 * al(n64);
  cudaError_t e = cudaStreamCreateWithFlags(&ws->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete ws;
    return cuda_error(e, "solver stream");
  }
  cudaStream_t s = ws->stream;
  e = cudaMallocAsync(&ws->base, total, s);
  if (e != cudaSuccess) {
    cudaStreamDestroy(s);
    delete ws;
    return set_error(MFX_ENOMEM, "solver workspace allocation failed");
  }
  ws->h_st = pinned_status_get();
  if (!ws->h_st) {
    cudaFreeAsync(ws->base, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    delete ws;
    return set_error(MFX_ENOMEM, "pinned status allocation failed");
  }
  char* p = (char*)ws->base;
  ws->st = (SolveState*)p;
  p += al(sizeof(SolveState));
  ws->scal = (double*)p;
  p += al(64 * sizeof(double));
  if (op->has_f64) {
    double** f[] = {&ws->w64.x, &ws->w64.r, &ws->w64.p, &ws->w64.q, &ws->w64.z,
                    &ws->w64.d, &ws->w64.t, &ws->w64.dinv, &ws->w64.b};
    for (auto* v : f) {
      *v = (double*)p;
      p += al(n64);
    }
  }
  if (op->has_f32) {
    float** f[] = {&ws->w32.x, &ws->w32.r, &ws->w32.p, &ws->w32.q, &ws->w32.z,
                   &ws->w32.d, &ws->w32.t, &ws->w32.dinv, &ws->w32.b};
    for (auto* v : f) {
      *v = (float*)p;
      p += al(n32);
    }
    ws->r64 = (double*)p;
    p += al(n64);
    ws->y64 = (double*)p;
    p += al(n64);
  }
  ws->bytes = total;
  op->d_work = ws;
  op->work_bytes = total;
  // inverse diagonals
  if (op->has_f64) reciprocal_kernel<double><<<vec_grid(n), 256, 0, s>>>(n, op->d_diag64, ws->w64.dinv);
  if (op->has_f32) reciprocal_kernel<float><<<vec_grid(n), 256, 0, s>>>(n, op->d_diag32, ws->w32.dinv);
  // one application per precision outside any capture (first-launch kernel attributes)
  if (op->has_f64) {
    MFX_CUDA_TRY(cudaMemsetAsync(ws->w64.p, 0, n64, s));
    mfx_status rc = launch_vmult(op, MFX_F64, ws->w64.p, ws->w64.q, s);
    if (rc != MFX_OK) return rc;
  }
  if (op->has_f32) {
    MFX_CUDA_TRY(cudaMemsetAsync(ws->w32.p, 0, n32, s));
    mfx_status rc = launch_vmult(op, MFX_F32, ws->w32.p, ws->w32.q, s);
    if (rc != MFX_OK) return rc;
  }
  MFX_CUDA_TRY(cudaStreamSynchronize(s));
  return MFX_OK;
}

// Frees the workspace in stream order on `s` (0: its own stream, after its pending work).
void free_workspace(mfx_op* op, cudaStream_t s) {
  auto* ws = workspace(op);
  if (!ws) return;
  cudaFreeAsync(ws->base, s ? s : ws->stream);
  pinned_status_put(ws->h_st);
  cudaStreamDestroy(ws->stream);  // returns at once; resources go when its work is done
  delete ws;
  op->d_work = nullptr;
  op->work_bytes = 0;
}

mfx_status prepare_workspace(mfx_op* op) { return ensure_workspace(op); }

template <typename Real>
static Work<Real>& work_of(SolveWorkspace* ws);
template <>
Work<double>& work_of<double>(SolveWorkspace* ws) { return ws->w64; }
template <>
Work<float>& work_of<float>(SolveWorkspace* ws) { return ws->w32; }

template <typename Real>
static constexpr mfx_prec prec_of() { return std::is_same<Real, double>::value ? MFX_F64 : MFX_F32; }

// z = Chebyshev(r); uses w.d and w.t; skip: optional done flag.
template <typename Real>
static mfx_status cheb_apply(const mfx_op* op, Work<Real>& w, const Real* r, Real* z, int degree, double lo,
                             double hi, const int32_t* skip, cudaStream_t s) {
  const int64_t n = op->n_dofs;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  cheb_init_kernel<Real><<<vec_grid(n), 256, 0, s>>>(n, r, w.dinv, w.d, z, (Real)(1.0 / theta), skip);
  for (int i = 1; i < degree; ++i) {
    mfx_status st = launch_vmult(op, prec_of<Real>(), z, w.t, s, skip);
    if (st != MFX_OK) return st;
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    cheb_step_kernel<Real><<<vec_grid(n), 256, 0, s>>>(n, r, w.t, w.dinv, w.d, z, (Real)(rho_new * rho),
                                                        (Real)(2.0 * rho_new / delta), skip);
    rho = rho_new;
  }
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

}  // namespace mfx

struct mfx_mg;

namespace mfx {

// Preconditioner of a PCG: Jacobi (fused into the CG update), Chebyshev(degree) in D^-1 K on
// [lo, hi], or the multigrid V-cycle of `mg` (mg.cuh).
struct Precond {
  int kind = 0;  // 0 Jacobi, 1 Chebyshev, 2 multigrid
  int degree = 0;
  double lo = 0.0, hi = 0.0;
  mfx_mg* mg = nullptr;
};

template <typename Real>
mfx_status mg_vcycle(mfx_mg* mg, const Real* r, Real* z, const int32_t* skip, cudaStream_t s);

template <typename Real>
static mfx_status precond_apply(const mfx_op* op, Work<Real>& w, const Precond& pc, const Real* r, Real* z,
                                const int32_t* skip, cudaStream_t s) {
  if (pc.kind == 1) return cheb_apply<Real>(op, w, r, z, pc.degree, pc.lo, pc.hi, skip, s);
  return mg_vcycle<Real>(pc.mg, r, z, skip, s);
}

// One PCG iteration (all kernels no-op once done).
template <typename Real>
static mfx_status pcg_iteration(const mfx_op* op, SolveWorkspace* ws, Work<Real>& w, const Precond& pc, cudaStream_t s) {
  const int64_t n = op->n_dofs;
  const int g = reduction_blocks(n);
  const int32_t* done = &ws->st->done;
  const bool jacobi = pc.kind == 0;
  mfx_status rc = launch_vmult(op, prec_of<Real>(), w.p, w.q, s, done);
  if (rc != MFX_OK) return rc;
  cg_pq_kernel<Real><<<g, kRedThreads, 0, s>>>(n, w.p, w.q, ws->st, op->d_partials, op->d_counter);
  cg_update_kernel<Real><<<g, kRedThreads, 0, s>>>(n, w.x, w.r, w.p, w.q, w.dinv, jacobi, ws->st, op->d_partials,
                                                   op->d_counter);
  if (!jacobi) {
    rc = precond_apply<Real>(op, w, pc, w.r, w.z, done, s);
    if (rc != MFX_OK) return rc;
    cg_rz_kernel<Real><<<g, kRedThreads, 0, s>>>(n, w.r, w.z, ws->st, op->d_partials, op->d_counter);
    cg_p_kernel<Real><<<vec_grid(n), 256, 0, s>>>(n, w.p, w.r, w.dinv, w.z, ws->st);
  } else {
    cg_p_kernel<Real><<<vec_grid(n), 256, 0, s>>>(n, w.p, w.r, w.dinv, nullptr, ws->st);
  }
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

// Solve K x = b in precision Real (b, x in w.b, w.x).  Returns the final state in ws->h_st.
template <typename Real>
static mfx_status pcg_run(const mfx_op* op, SolveWorkspace* ws, const Precond& pc, double tol, int max_it,
                          int check_every, bool record, cudaStream_t s) {
  Work<Real>& w = work_of<Real>(ws);
  const int64_t n = op->n_dofs;
  const int g = reduction_blocks(n);
  const bool jacobi = pc.kind == 0;
  SolveState init{};
  init.tol2 = tol * tol;
  init.max_it = max_it;
  init.record = record ? 1 : 0;
  MFX_CUDA_TRY(cudaMemcpyAsync(ws->st, &init, sizeof(SolveState), cudaMemcpyHostToDevice, s));
  cg_init_kernel<Real><<<g, kRedThreads, 0, s>>>(n, w.b, w.x, w.r, w.p, w.dinv, jacobi, ws->st, op->d_partials,
                                                 op->d_counter);
  if (!jacobi) {
    mfx_status rc = precond_apply<Real>(op, w, pc, w.r, w.p, &ws->st->done, s);
    if (rc != MFX_OK) return rc;
    // rz = (r, z) with z = p
    dot_kernel<Real><<<g, kRedThreads, 0, s>>>(n, w.r, w.p, &ws->st->rz, op->d_partials, op->d_counter);
  }
  MFX_CUDA_TRY(cudaGetLastError());
  // capture a chunk of iterations once, then replay it until done
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  MFX_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  mfx_status rc = MFX_OK;
  for (int i = 0; i < check_every && rc == MFX_OK; ++i) rc = pcg_iteration<Real>(op, ws, w, pc, s);
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (rc != MFX_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphInstantiate");
  int launched = 0;
  for (;;) {
    ce = cudaGraphLaunch(exec, s);
    if (ce != cudaSuccess) break;
    launched += check_every;
    ce = cudaMemcpyAsync(ws->h_st, ws->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) break;
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) break;
    if (ws->h_st->done || launched >= max_it + check_every) break;
  }
  cudaGraphExecDestroy(exec);
  if (ce != cudaSuccess) return cuda_error(ce, "pcg loop");
  return MFX_OK;
}

// Largest eigenvalue of a symmetric tridiagonal matrix by Sturm-sequence bisection.
static double tridiag_lambda_max(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // number of eigenvalues < x
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      q = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) < m)
      lo = mid;
    else
      hi = mid;
    if (hi - lo <= 1e-15 * std::fabs(hi)) break;
  }
  return hi;
}

template <typename Real>
static mfx_status estimate_lambda(const mfx_op* op, SolveWorkspace* ws, const double* start, int steps,
                                  cudaStream_t s, double* lam) {
  Work<Real>& w = work_of<Real>(ws);
  const int64_t n = op->n_dofs;
  steps = std::max(2, std::min(steps, kMaxLanczos - 1));
  convert_kernel<Real><<<vec_grid(n), 256, 0, s>>>(n, start, w.b);
  // constrained rows do not belong to D^-1 K on the free space: zero them
  mfx_status rc = pcg_run<Real>(op, ws, Precond{}, 0.0, steps, steps, true, s);
  if (rc != MFX_OK) return rc;
  const SolveState& h = *ws->h_st;
  const int m = std::min(h.it, steps);
  if (m < 1) return set_error(MFX_BREAKDOWN, "eigenvalue estimate: no CG step");
  std::vector<double> a(m), b(std::max(0, m - 1));
  for (int i = 0; i < m; ++i) {
    a[i] = 1.0 / h.lan_alpha[i] + (i > 0 ? h.lan_beta[i - 1] / h.lan_alpha[i - 1] : 0.0);
    if (i + 1 < m) b[i] = std::sqrt(h.lan_beta[i]) / h.lan_alpha[i];
  }
  *lam = tridiag_lambda_max(a, b);
  return MFX_OK;
}

}  // namespace mfx

extern "C" void mfx_solve_params_default(mfx_solve_params* p);

namespace mfx {

// PCG (Jacobi or Chebyshev-Jacobi, or the V-cycle of mg when mg is not null) in FP64, or FP64
// defect correction around the FP32 PCG (mixed).
mfx_status solve_impl(mfx_op* op, const double* b, double* x, const mfx_solve_params* params, mfx_mg* mg,
                      mfx_solve_stats* stats, mfx_stream stream) {
  if (!op || !b || !x || !stats) return set_error(MFX_EINVAL, "mfx_solve: null argument");
  const auto t_start = std::chrono::steady_clock::now();
  mfx_solve_params p;
  mfx_solve_params_default(&p);
  if (params) p = *params;
  if (!(p.tol >= 0.0) || p.max_it < 1 || p.cheb_degree < 1 || (p.precond != MFX_PRECOND_JACOBI && p.precond != MFX_PRECOND_CHEBYSHEV))
    return set_error(MFX_EINVAL, "mfx_solve: bad parameters");
  const bool mixed = p.mixed != 0;
  if (mixed && !(op->has_f32 && op->has_f64))
    return set_error(MFX_EINVAL, "mfx_solve: mixed precision needs FP64 and FP32 data");
  if (!mixed && !op->has_f64) return set_error(MFX_EINVAL, "mfx_solve: FP64 data not built");
  mfx_status rc = ensure_workspace(op);
  if (rc != MFX_OK) return rc;
  auto* ws = workspace(op);
  // order after the caller's work, then run on the solver stream (capturable)
  MFX_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  cudaStream_t s = ws->stream;
  const int64_t n = op->n_dofs;
  const int g = reduction_blocks(n);
  const bool cheb = !mg && p.precond == MFX_PRECOND_CHEBYSHEV;
  const int check = p.check_every > 0 ? p.check_every : 8;
  *stats = mfx_solve_stats{};
  const int pi = mixed ? 1 : 0;
  double lo = p.cheb_lo, hi = p.cheb_hi;
  if (cheb && !(hi > 0.0)) {
    if (ws->lambda_max[pi] == 0.0 || p.lanczos_start) {
      double lam = 0.0;
      const double* start = p.lanczos_start ? p.lanczos_start : b;
      rc = mixed ? estimate_lambda<float>(op, ws, start, p.lanczos_steps, s, &lam)
                 : estimate_lambda<double>(op, ws, start, p.lanczos_steps, s, &lam);
      if (rc != MFX_OK) return rc;
      ws->lambda_max[pi] = lam;
    }
    stats->lambda_max = ws->lambda_max[pi];
    hi = 1.2 * ws->lambda_max[pi];
    lo = hi / 20.0;
  }
  stats->cheb_lo = lo;
  stats->cheb_hi = hi;
  Precond pc;
  pc.kind = mg ? 2 : (cheb ? 1 : 0);
  pc.degree = p.cheb_degree;
  pc.lo = lo;
  pc.hi = hi;
  pc.mg = mg;
  if (!mixed) {
    MFX_CUDA_TRY(cudaMemcpyAsync(ws->w64.b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    rc = pcg_run<double>(op, ws, pc, p.tol, p.max_it, check, false, s);
    if (rc != MFX_OK) return rc;
    stats->iterations = ws->h_st->it;
    stats->status = ws->h_st->status;
    MFX_CUDA_TRY(cudaMemcpyAsync(x, ws->w64.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    MFX_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    double* rr = ws->scal;      // (r, r)
    double* bb = ws->scal + 1;  // (b, b)
    double h[2];
    launch_dot(op, MFX_F64, n, b, b, bb, s);
    stats->status = MFX_NOT_CONVERGED;
    int inner_total = 0;
    for (int outer = 0; outer <= p.max_it; ++outer) {
      rc = launch_vmult(op, MFX_F64, x, ws->y64, s);
      if (rc != MFX_OK) return rc;
      residual_kernel<<<g, kRedThreads, 0, s>>>(n, b, ws->y64, ws->r64, rr, op->d_partials, op->d_counter);
      MFX_CUDA_TRY(cudaMemcpyAsync(h, ws->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      MFX_CUDA_TRY(cudaStreamSynchronize(s));
      stats->iterations = outer;
      if (!std::isfinite(h[0])) {
        stats->status = MFX_BREAKDOWN;
        break;
      }
      if (h[0] <= p.tol * p.tol * h[1]) {
        stats->status = MFX_OK;
        break;
      }
      if (outer == p.max_it) break;
      scale_to_f32_kernel<<<vec_grid(n), 256, 0, s>>>(n, ws->r64, rr, ws->w32.b);
      rc = pcg_run<float>(op, ws, pc, p.inner_tol, p.inner_max_it, check, false, s);
      if (rc != MFX_OK) return rc;
      inner_total += ws->h_st->it;
      if (ws->h_st->status == MFX_BREAKDOWN) {
        stats->status = MFX_BREAKDOWN;
        break;
      }
      add_scaled_f32_kernel<<<vec_grid(n), 256, 0, s>>>(n, x, ws->w32.x, rr);
    }
    stats->inner_iterations = inner_total;
  }
  // true FP64 residual of the result
  rc = launch_vmult(op, MFX_F64, x, ws->y64 ? ws->y64 : ws->w64.q, s);
  if (rc != MFX_OK) return rc;
  double* rr = ws->scal + 2;
  double* bb = ws->scal + 3;
  residual_kernel<<<g, kRedThreads, 0, s>>>(n, b, ws->y64 ? ws->y64 : ws->w64.q, ws->r64 ? ws->r64 : ws->w64.t, rr,
                                            op->d_partials, op->d_counter);
  launch_dot(op, MFX_F64, n, b, b, bb, s);
  double h[2];
  MFX_CUDA_TRY(cudaMemcpyAsync(h, rr, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MFX_CUDA_TRY(cudaStreamSynchronize(s));
  stats->rel_residual = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
  stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return MFX_OK;
}


}  // namespace mfx

using namespace mfx;

extern "C" {

void mfx_solve_params_default(mfx_solve_params* p) {
  if (!p) return;
  p->tol = 1e-10;
  p->max_it = 100000;
  p->precond = MFX_PRECOND_JACOBI;
  p->cheb_degree = 5;
  p->mixed = 0;
  p->inner_tol = 1e-4;
  p->check_every = 0;
  p->lanczos_steps = 15;
  p->cheb_lo = 0.0;
  p->cheb_hi = 0.0;
  p->lanczos_start = nullptr;
  p->inner_max_it = 10000;
  p->reserved = 0;
}

mfx_status mfx_dot(const mfx_op* op, mfx_prec prec, int64_t n, const void* a, const void* b, double* result,
                   mfx_stream stream) {
  if (!op || !a || !b || !result || n < 0 || (prec != MFX_F64 && prec != MFX_F32))
    return set_error(MFX_EINVAL, "mfx_dot: bad arguments");
  return launch_dot(op, prec, n, a, b, result, (cudaStream_t)stream);
}

mfx_status mfx_chebyshev(const mfx_op* op_c, mfx_prec prec, const void* r, void* z, int32_t degree, double lo,
                         double hi, mfx_stream stream) {
  mfx_op* op = const_cast<mfx_op*>(op_c);
  if (!op || !r || !z || degree < 1 || !(hi > lo) || !(lo > 0.0))
    return set_error(MFX_EINVAL, "mfx_chebyshev: bad arguments");
  if ((prec == MFX_F64 && !op->has_f64) || (prec == MFX_F32 && !op->has_f32))
    return set_error(MFX_EINVAL, "mfx_chebyshev: precision not built for this operator");
  mfx_status rc = ensure_workspace(op);
  if (rc != MFX_OK) return rc;
  auto* ws = workspace(op);
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == MFX_F64) return cheb_apply<double>(op, ws->w64, (const double*)r, (double*)z, degree, lo, hi, nullptr, s);
  return cheb_apply<float>(op, ws->w32, (const float*)r, (float*)z, degree, lo, hi, nullptr, s);
}

mfx_status mfx_solve(const mfx_op* op_c, const double* b, double* x, const mfx_solve_params* params,
                     mfx_solve_stats* stats, mfx_stream stream) {
  MFX_TRACE("mfx_solve");
  return solve_impl(const_cast<mfx_op*>(op_c), b, x, params, nullptr, stats, stream);
}

}  // extern "C"

// ------------------------------------------------------------------ batches of solves
//
// A batch holds up to max_slots independent solves (one operator each).  A slot runs the
// mixed-precision solve as a state machine: OUTER (FP64 residual b - K64 x and its norm; stop or
// start an inner solve on r / ||r||), INNER (FP32 PCG, advanced `chunk` iterations per tick by a
// captured graph), then x += ||r|| d and back to OUTER.  With mixed = 0 the INNER phase is the FP64
// PCG on b itself.  Every tick launches one parent graph whose child nodes are the chunk graphs of
// all slots in the INNER phase, so all active problems advance together and overlap on the GPU;
// converged problems leave their slot, new problems can be added between ticks.

namespace mfx {

enum { SLOT_FREE = 0, SLOT_OUTER = 1, SLOT_INNER = 2, SLOT_DONE = 3 };

struct BatchSlot {
  mfx_op* op = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  mfx_solve_params p{};
  int phase = SLOT_FREE;
  bool mixed = true, cheb = false;
  double lo = 0, hi = 0, bb = 0, rr = 0;
  int outer = 0, inner_total = 0, status = MFX_OK;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;  // one chunk of inner iterations (ends with a copy of the state to the host)
  cudaGraphExec_t exec = nullptr;  // the same chunk, for independent (asynchronous) stepping
  cudaEvent_t event = nullptr;     // completion of the slot's last launched work
  bool busy = false;               // work in flight (asynchronous stepping)
  bool residual_pending = false;   // OUTER: residual launched, norm not read yet
  bool bb_pending = true;          // (b, b) copied to h_scal[1] by the slot's stream, not read yet
  double* h_scal = nullptr;     // pinned: (r, r), (b, b)
};

}  // namespace mfx

struct mfx_batch {
  std::vector<mfx::BatchSlot> slots;
  int chunk = 8;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t parent = nullptr;
  std::vector<int> parent_members;
  int64_t ticks = 0;
  void* run_state = nullptr;  // device RunState per slot (mfx_batch_run), allocated at the first run
  int64_t runs = 0;
};

namespace mfx {

static void slot_release(BatchSlot& sl) {
  if (sl.exec) cudaGraphExecDestroy(sl.exec);
  sl.exec = nullptr;
  if (sl.graph) cudaGraphDestroy(sl.graph);
  sl.graph = nullptr;
  sl.busy = false;
  sl.residual_pending = false;
  sl.op = nullptr;
  sl.phase = SLOT_FREE;
}

// (b, b) of a slot, once the slot's stream has passed the copy queued by mfx_batch_add.
static void slot_read_bb(BatchSlot& sl) {
  if (!sl.bb_pending) return;
  sl.bb = sl.h_scal[1];
  sl.bb_pending = false;
}

// Decision after the FP64 residual of an OUTER slot: done, or start the next inner solve.
static mfx_status slot_outer_decide(BatchSlot& sl, bool* start_inner) {
  slot_read_bb(sl);
  sl.rr = sl.h_scal[0];
  *start_inner = false;
  if (!std::isfinite(sl.rr) || !std::isfinite(sl.bb)) {
    sl.phase = SLOT_DONE;
    sl.status = MFX_BREAKDOWN;
  } else if (sl.rr <= sl.p.tol * sl.p.tol * sl.bb) {
    sl.phase = SLOT_DONE;
    sl.status = MFX_OK;
  } else if (sl.outer >= sl.p.max_it) {
    sl.phase = SLOT_DONE;
    sl.status = MFX_NOT_CONVERGED;
  } else {
    *start_inner = true;
  }
  return MFX_OK;
}

// Capture one chunk of inner PCG iterations of the slot's operator.
template <typename Real>
static mfx_status capture_chunk(BatchSlot& sl, int chunk) {
  SolveWorkspace* ws = workspace(sl.op);
  Work<Real>& w = work_of<Real>(ws);
  cudaGraph_t g = nullptr;
  MFX_CUDA_TRY(cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal));
  mfx_status rc = MFX_OK;
  for (int i = 0; i < chunk && rc == MFX_OK; ++i)
    rc = pcg_iteration<Real>(sl.op, ws, w, Precond{sl.cheb ? 1 : 0, sl.p.cheb_degree, sl.lo, sl.hi, nullptr},
                             sl.stream);
  cudaMemcpyAsync(ws->h_st, ws->st, sizeof(SolveState), cudaMemcpyDeviceToHost, sl.stream);
  cudaError_t ce = cudaStreamEndCapture(sl.stream, &g);
  if (rc != MFX_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ce != cudaSuccess) return cuda_error(ce, "batch chunk capture");
  sl.graph = g;
  ce = cudaGraphInstantiate(&sl.exec, g, 0);
  if (ce != cudaSuccess) return cuda_error(ce, "batch chunk instantiate");
  return MFX_OK;
}

// Start an inner solve: FP32 on r / ||r|| (mixed) or FP64 on b.
static mfx_status slot_start_inner(BatchSlot& sl) {
  SolveWorkspace* ws = workspace(sl.op);
  const int64_t n = sl.op->n_dofs;
  const int g = reduction_blocks(n);
  SolveState init{};
  init.tol2 = sl.mixed ? sl.p.inner_tol * sl.p.inner_tol : sl.p.tol * sl.p.tol;
  init.max_it = sl.mixed ? sl.p.inner_max_it : sl.p.max_it;
  MFX_CUDA_TRY(cudaMemcpyAsync(ws->st, &init, sizeof(SolveState), cudaMemcpyHostToDevice, sl.stream));
  if (sl.mixed) {
    scale_to_f32_kernel<<<vec_grid(n), 256, 0, sl.stream>>>(n, ws->r64, ws->scal, ws->w32.b);
    cg_init_kernel<float><<<g, kRedThreads, 0, sl.stream>>>(n, ws->w32.b, ws->w32.x, ws->w32.r, ws->w32.p,
                                                            ws->w32.dinv, !sl.cheb, ws->st, sl.op->d_partials,
                                                            sl.op->d_counter);
    if (sl.cheb) {
      mfx_status rc = cheb_apply<float>(sl.op, ws->w32, ws->w32.r, ws->w32.p, sl.p.cheb_degree, sl.lo, sl.hi,
                                        &ws->st->done, sl.stream);
      if (rc != MFX_OK) return rc;
      dot_kernel<float><<<g, kRedThreads, 0, sl.stream>>>(n, ws->w32.r, ws->w32.p, &ws->st->rz, sl.op->d_partials,
                                                          sl.op->d_counter);
    }
  } else {
    MFX_CUDA_TRY(cudaMemcpyAsync(ws->w64.b, sl.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, sl.stream));
    cg_init_kernel<double><<<g, kRedThreads, 0, sl.stream>>>(n, ws->w64.b, ws->w64.x, ws->w64.r, ws->w64.p,
                                                             ws->w64.dinv, !sl.cheb, ws->st, sl.op->d_partials,
                                                             sl.op->d_counter);
    if (sl.cheb) {
      mfx_status rc = cheb_apply<double>(sl.op, ws->w64, ws->w64.r, ws->w64.p, sl.p.cheb_degree, sl.lo, sl.hi,
                                         &ws->st->done, sl.stream);
      if (rc != MFX_OK) return rc;
      dot_kernel<double><<<g, kRedThreads, 0, sl.stream>>>(n, ws->w64.r, ws->w64.p, &ws->st->rz,
                                                           sl.op->d_partials, sl.op->d_counter);
    }
  }
  MFX_CUDA_TRY(cudaGetLastError());
  sl.phase = SLOT_INNER;
  return MFX_OK;
}

// Launch the FP64 residual of an OUTER slot (result read after the tick's synchronisation).
static mfx_status slot_launch_residual(BatchSlot& sl) {
  SolveWorkspace* ws = workspace(sl.op);
  const int64_t n = sl.op->n_dofs;
  mfx_status rc = launch_vmult(sl.op, MFX_F64, sl.x, ws->y64, sl.stream);
  if (rc != MFX_OK) return rc;
  residual_kernel<<<reduction_blocks(n), kRedThreads, 0, sl.stream>>>(n, sl.b, ws->y64, ws->r64, ws->scal,
                                                                      sl.op->d_partials, sl.op->d_counter);
  MFX_CUDA_TRY(cudaMemcpyAsync(sl.h_scal, ws->scal, sizeof(double), cudaMemcpyDeviceToHost, sl.stream));
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

static mfx_status rebuild_parent(mfx_batch* bt) {
  std::vector<int> members;
  for (size_t i = 0; i < bt->slots.size(); ++i)
    if (bt->slots[i].phase == SLOT_INNER) members.push_back((int)i);
  if (bt->parent && members == bt->parent_members) return MFX_OK;
  if (bt->parent) cudaGraphExecDestroy(bt->parent);
  bt->parent = nullptr;
  bt->parent_members = members;
  if (members.empty()) return MFX_OK;
  cudaGraph_t g = nullptr;
  MFX_CUDA_TRY(cudaGraphCreate(&g, 0));
  for (int i : members) {
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, bt->slots[i].graph);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_error(e, "cudaGraphAddChildGraphNode");
    }
  }
  cudaError_t e = cudaGraphInstantiate(&bt->parent, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate (batch)");
  return MFX_OK;
}

// ------------------------------------------------------------------ whole solves in one launch
//
// mfx_batch_run builds one graph that holds every active slot's complete solve and launches it once.
// The loops are graph WHILE nodes whose conditions kernels set on the device: the outer loop of the
// mixed solve (FP64 residual, stopping test, FP32 inner solve, correction) and, nested in it, the
// inner PCG loop (a chunk of iterations, then the test of the inner state).  The device decides when
// each problem stops; the host only builds the graph and reads the states afterwards.  Every loop
// condition kernel also counts its passes and ends the loop beyond a cap (max_it for the outer loop,
// inner_max_it / chunk + 2 chunks for the inner one), so every loop ends.

struct RunState {
  double bb, rr;  // (b, b) and the last FP64 (r, r)
  int32_t outer, inner_total, status, done;
  int32_t inner_passes, outer_passes;
};

// start of a slot's run: (b, b) from the value mfx_batch_add computed; outer loop on
__global__ void run_start_kernel(RunState* rs, const double* bb, cudaGraphConditionalHandle outer) {
  rs->bb = *bb;
  rs->rr = 0.0;
  rs->outer = 0;
  rs->inner_total = 0;
  rs->status = MFX_NOT_CONVERGED;
  rs->done = 0;
  rs->inner_passes = 0;
  rs->outer_passes = 0;
  cudaGraphSetConditional(outer, 1u);
}

// mixed solve, top of an outer pass: stopping test on the FP64 residual; otherwise the inner solve's
// state is reset (tolerance and cap of the inner solve) and its loop switched on
__global__ void run_decide_kernel(RunState* rs, SolveState* st, double tol2, int max_outer, double inner_tol2,
                                  int inner_max_it, cudaGraphConditionalHandle outer, cudaGraphConditionalHandle inner) {
  const double rr = rs->rr, bb = rs->bb;
  rs->outer_passes += 1;
  int done = 0;
  if (!isfinite(rr) || !isfinite(bb)) {
    rs->status = MFX_BREAKDOWN;
    done = 1;
  } else if (rr <= tol2 * bb) {
    rs->status = MFX_OK;
    done = 1;
  } else if (rs->outer >= max_outer || rs->outer_passes > max_outer + 1) {
    rs->status = MFX_NOT_CONVERGED;
    done = 1;
  }
  rs->done = done;
  rs->inner_passes = 0;
  st->tol2 = inner_tol2;
  st->max_it = inner_max_it;
  st->record = 0;
  st->it = 0;
  st->done = done;  // the inner solve's kernels do nothing for a finished slot
  cudaGraphSetConditional(outer, done ? 0u : 1u);
  cudaGraphSetConditional(inner, done ? 0u : 1u);
}

// inner loop test after a chunk of PCG iterations
__global__ void run_inner_check_kernel(RunState* rs, const SolveState* st, int max_passes,
                                       cudaGraphConditionalHandle inner) {
  rs->inner_passes += 1;
  cudaGraphSetConditional(inner, (!st->done && rs->inner_passes < max_passes) ? 1u : 0u);
}

// FP32 start of the inner solve on r / ||r|| (skipped for a finished slot)
__global__ void run_scale_kernel(int64_t n, const double* __restrict__ r, const RunState* rs,
                                 float* __restrict__ out) {
  if (rs->done) return;
  const double sc = 1.0 / sqrt(rs->rr);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)(r[i] * sc);
}

// x += ||r|| d after an inner solve that did not break down (skipped for a finished slot)
__global__ void run_correct_kernel(int64_t n, double* __restrict__ x, const float* __restrict__ d,
                                   const RunState* rs, const SolveState* st) {
  if (rs->done || st->status == MFX_BREAKDOWN) return;
  const double sc = sqrt(rs->rr);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += sc * (double)d[i];
}

// end of an outer pass: count the inner iterations; an inner breakdown ends the slot
__global__ void run_advance_kernel(RunState* rs, const SolveState* st, cudaGraphConditionalHandle outer) {
  if (rs->done) return;
  rs->inner_total += st->it;
  if (st->status == MFX_BREAKDOWN) {
    rs->status = MFX_BREAKDOWN;
    rs->done = 1;
    cudaGraphSetConditional(outer, 0u);
    return;
  }
  rs->outer += 1;
}

// FP64 solve: the PCG state before its start kernel
__global__ void run_state64_kernel(SolveState* st, double tol2, int max_it) {
  st->tol2 = tol2;
  st->max_it = max_it;
  st->record = 0;
  st->it = 0;
  st->done = 0;
  st->status = MFX_OK;
}

// FP64 solve: final state of the PCG
__global__ void run_finish64_kernel(RunState* rs, const SolveState* st) {
  rs->status = st->status;
  rs->inner_total = st->it;
  rs->rr = st->rr;
  rs->done = 1;
}

// Appends what `body` launches on stream s to graph g after the nodes deps[0..nd), and returns the
// captured work's last node in *leaf (or the first dependency if nothing was captured).
template <typename F>
static mfx_status capture_segment(cudaStream_t s, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                  cudaGraphNode_t* leaf, F&& body) {
  MFX_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, deps, nullptr, nd, cudaStreamCaptureModeThreadLocal));
  mfx_status rc = body();
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* out = nullptr;
  size_t n_out = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &out, nullptr, &n_out);
  cudaGraphNode_t last = (e == cudaSuccess && n_out > 0) ? out[n_out - 1] : (nd > 0 ? deps[0] : nullptr);
  const size_t n_leaves = n_out;
  cudaGraph_t tmp = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &tmp);
  if (rc != MFX_OK) return rc;
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamGetCaptureInfo");
  if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamEndCapture (segment)");
  if (n_leaves > 1) return set_error(MFX_ECUDA, "batch run: a captured segment ended in several nodes");
  *leaf = last;
  return MFX_OK;
}

static mfx_status add_while(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h, cudaGraphNode_t* node,
                            cudaGraph_t* body) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  MFX_CUDA_TRY(cudaGraphAddNode(node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &p));
  *body = p.conditional.phGraph_out[0];
  return MFX_OK;
}

// The inner PCG loop of a slot (precision Real) after node dep of graph g: WHILE(inner) { chunk of
// iterations; test }.  The loop's condition must be set upstream.
template <typename Real>
static mfx_status add_inner_loop(BatchSlot& sl, int chunk, RunState* rs, cudaGraph_t g, cudaGraphNode_t dep,
                                 cudaGraphConditionalHandle inner, cudaGraphNode_t* node) {
  SolveWorkspace* ws = workspace(sl.op);
  Work<Real>& w = work_of<Real>(ws);
  cudaGraph_t body = nullptr;
  mfx_status rc = add_while(g, dep, inner, node, &body);
  if (rc != MFX_OK) return rc;
  const int max_it = sl.mixed ? sl.p.inner_max_it : sl.p.max_it;
  const int max_passes = max_it / chunk + 2;
  const Precond pc{sl.cheb ? 1 : 0, sl.p.cheb_degree, sl.lo, sl.hi, nullptr};
  cudaGraphNode_t leaf = nullptr;
  return capture_segment(sl.stream, body, nullptr, 0, &leaf, [&]() -> mfx_status {
    for (int i = 0; i < chunk; ++i) {
      mfx_status r2 = pcg_iteration<Real>(sl.op, ws, w, pc, sl.stream);
      if (r2 != MFX_OK) return r2;
    }
    run_inner_check_kernel<<<1, 1, 0, sl.stream>>>(rs, ws->st, max_passes, inner);
    MFX_CUDA_TRY(cudaGetLastError());
    return MFX_OK;
  });
}

// One slot's whole solve, appended to graph g (no edges to other slots).
static mfx_status add_slot_solve(BatchSlot& sl, int chunk, RunState* rs, cudaGraph_t g) {
  SolveWorkspace* ws = workspace(sl.op);
  const int64_t n = sl.op->n_dofs;
  const int red = reduction_blocks(n);
  cudaStream_t s = sl.stream;
  if (!sl.mixed) {
    // FP64 PCG on b: start, loop, copy the solution out
    cudaGraphConditionalHandle inner;
    MFX_CUDA_TRY(cudaGraphConditionalHandleCreate(&inner, g, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t start = nullptr, loop = nullptr, fin = nullptr;
    mfx_status rc = capture_segment(s, g, nullptr, 0, &start, [&]() -> mfx_status {
      run_start_kernel<<<1, 1, 0, s>>>(rs, ws->scal + 1, inner);  // the start sets this loop's condition
      run_state64_kernel<<<1, 1, 0, s>>>(ws->st, sl.p.tol * sl.p.tol, sl.p.max_it);
      MFX_CUDA_TRY(cudaMemcpyAsync(ws->w64.b, sl.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      cg_init_kernel<double><<<red, kRedThreads, 0, s>>>(n, ws->w64.b, ws->w64.x, ws->w64.r, ws->w64.p, ws->w64.dinv,
                                                         !sl.cheb, ws->st, sl.op->d_partials, sl.op->d_counter);
      if (sl.cheb) {
        mfx_status r2 = cheb_apply<double>(sl.op, ws->w64, ws->w64.r, ws->w64.p, sl.p.cheb_degree, sl.lo, sl.hi,
                                           &ws->st->done, s);
        if (r2 != MFX_OK) return r2;
        dot_kernel<double><<<red, kRedThreads, 0, s>>>(n, ws->w64.r, ws->w64.p, &ws->st->rz, sl.op->d_partials,
                                                       sl.op->d_counter);
      }
      MFX_CUDA_TRY(cudaGetLastError());
      return MFX_OK;
    });
    if (rc != MFX_OK) return rc;
    rc = add_inner_loop<double>(sl, chunk, rs, g, start, inner, &loop);
    if (rc != MFX_OK) return rc;
    return capture_segment(s, g, &loop, 1, &fin, [&]() -> mfx_status {
      MFX_CUDA_TRY(cudaMemcpyAsync(sl.x, ws->w64.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      run_finish64_kernel<<<1, 1, 0, s>>>(rs, ws->st);
      MFX_CUDA_TRY(cudaGetLastError());
      return MFX_OK;
    });
  }
  // mixed: WHILE(outer) { residual, decide; scale, FP32 PCG start; WHILE(inner) {...}; correct, advance }
  cudaGraphConditionalHandle outer;
  MFX_CUDA_TRY(cudaGraphConditionalHandleCreate(&outer, g, 0, cudaGraphCondAssignDefault));
  cudaGraphNode_t start = nullptr, oloop = nullptr;
  mfx_status rc = capture_segment(s, g, nullptr, 0, &start, [&]() -> mfx_status {
    // a mixed solve starts from x = 0 (a slot that was stepped before starts over)
    MFX_CUDA_TRY(cudaMemsetAsync(sl.x, 0, sizeof(double) * n, s));
    run_start_kernel<<<1, 1, 0, s>>>(rs, ws->scal + 1, outer);
    MFX_CUDA_TRY(cudaGetLastError());
    return MFX_OK;
  });
  if (rc != MFX_OK) return rc;
  cudaGraph_t obody = nullptr;
  rc = add_while(g, start, outer, &oloop, &obody);
  if (rc != MFX_OK) return rc;
  cudaGraphConditionalHandle inner;
  MFX_CUDA_TRY(cudaGraphConditionalHandleCreate(&inner, obody, 0, cudaGraphCondAssignDefault));
  cudaGraphNode_t head = nullptr, iloop = nullptr, tail = nullptr;
  rc = capture_segment(s, obody, nullptr, 0, &head, [&]() -> mfx_status {
    mfx_status r2 = launch_vmult(sl.op, MFX_F64, sl.x, ws->y64, s);
    if (r2 != MFX_OK) return r2;
    residual_kernel<<<red, kRedThreads, 0, s>>>(n, sl.b, ws->y64, ws->r64, &rs->rr, sl.op->d_partials,
                                                sl.op->d_counter);
    run_decide_kernel<<<1, 1, 0, s>>>(rs, ws->st, sl.p.tol * sl.p.tol, sl.p.max_it, sl.p.inner_tol * sl.p.inner_tol,
                                      sl.p.inner_max_it, outer, inner);
    run_scale_kernel<<<vec_grid(n), 256, 0, s>>>(n, ws->r64, rs, ws->w32.b);
    cg_init_kernel<float><<<red, kRedThreads, 0, s>>>(n, ws->w32.b, ws->w32.x, ws->w32.r, ws->w32.p, ws->w32.dinv,
                                                      !sl.cheb, ws->st, sl.op->d_partials, sl.op->d_counter);
    if (sl.cheb) {
      r2 = cheb_apply<float>(sl.op, ws->w32, ws->w32.r, ws->w32.p, sl.p.cheb_degree, sl.lo, sl.hi, &ws->st->done, s);
      if (r2 != MFX_OK) return r2;
      dot_kernel<float><<<red, kRedThreads, 0, s>>>(n, ws->w32.r, ws->w32.p, &ws->st->rz, sl.op->d_partials,
                                                    sl.op->d_counter);
    }
    MFX_CUDA_TRY(cudaGetLastError());
    return MFX_OK;
  });
  if (rc != MFX_OK) return rc;
  rc = add_inner_loop<float>(sl, chunk, rs, obody, head, inner, &iloop);
  if (rc != MFX_OK) return rc;
  return capture_segment(s, obody, &iloop, 1, &tail, [&]() -> mfx_status {
    run_correct_kernel<<<vec_grid(n), 256, 0, s>>>(n, sl.x, ws->w32.x, rs, ws->st);
    run_advance_kernel<<<1, 1, 0, s>>>(rs, ws->st, outer);
    MFX_CUDA_TRY(cudaGetLastError());
    return MFX_OK;
  });
}

}  // namespace mfx

extern "C" {

mfx_status mfx_batch_create(mfx_batch** out, int32_t max_slots, int32_t chunk) try {
  if (!out || max_slots < 1 || max_slots > 4096) return set_error(MFX_EINVAL, "mfx_batch_create: bad arguments");
  *out = nullptr;
  auto* bt = new (std::nothrow) mfx_batch();
  if (!bt) return set_error(MFX_ENOMEM, "mfx_batch_create: host allocation failed");
  bt->slots.resize(max_slots);
  bt->chunk = chunk > 0 ? chunk : 8;
  cudaError_t e = cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking);
  for (auto& sl : bt->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_scal, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    mfx_batch_destroy(bt);
    return cuda_error(e, "mfx_batch_create");
  }
  *out = bt;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

void mfx_batch_destroy(mfx_batch* bt) {
  if (!bt) return;
  for (auto& sl : bt->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  if (bt->parent) cudaGraphExecDestroy(bt->parent);
  for (auto& sl : bt->slots) {
    slot_release(sl);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.event) cudaEventDestroy(sl.event);
    if (sl.h_scal) cudaFreeHost(sl.h_scal);
  }
  if (bt->stream) cudaStreamDestroy(bt->stream);
  if (bt->run_state) cudaFree(bt->run_state);
  delete bt;
}

mfx_status mfx_batch_add(mfx_batch* bt, const mfx_op* op_c, const double* b, double* x,
                         const mfx_solve_params* params, int32_t* slot_out) try {
  mfx_op* op = const_cast<mfx_op*>(op_c);
  if (!bt || !op || !b || !x || !slot_out) return set_error(MFX_EINVAL, "mfx_batch_add: null argument");
  mfx_solve_params p;
  mfx_solve_params_default(&p);
  if (params) p = *params;
  const bool mixed = p.mixed != 0;
  if (mixed && !(op->has_f32 && op->has_f64)) return set_error(MFX_EINVAL, "mixed solves need FP64 and FP32 data");
  if (!op->has_f64) return set_error(MFX_EINVAL, "batch solves need FP64 data");
  int free_slot = -1;
  for (size_t i = 0; i < bt->slots.size(); ++i) {
    if (bt->slots[i].phase != SLOT_FREE && bt->slots[i].op == op)
      return set_error(MFX_EBUSY, "operator already has an active slot");
    if (free_slot < 0 && bt->slots[i].phase == SLOT_FREE) free_slot = (int)i;
  }
  if (free_slot < 0) return set_error(MFX_EBUSY, "no free slot");
  mfx_status rc = ensure_workspace(op);
  if (rc != MFX_OK) return rc;
  BatchSlot& sl = bt->slots[free_slot];
  sl.op = op;
  sl.b = b;
  sl.x = x;
  sl.p = p;
  sl.mixed = mixed;
  sl.cheb = p.precond == MFX_PRECOND_CHEBYSHEV;
  sl.outer = 0;
  sl.inner_total = 0;
  sl.status = MFX_OK;
  SolveWorkspace* ws = workspace(op);
  if (sl.cheb) {
    const int pi = mixed ? 1 : 0;
    if (ws->lambda_max[pi] == 0.0) {
      double lam = 0.0;
      const double* start = p.lanczos_start ? p.lanczos_start : b;
      rc = mixed ? estimate_lambda<float>(op, ws, start, p.lanczos_steps, ws->stream, &lam)
                 : estimate_lambda<double>(op, ws, start, p.lanczos_steps, ws->stream, &lam);
      if (rc != MFX_OK) return rc;
      ws->lambda_max[pi] = lam;
    }
    sl.hi = p.cheb_hi > 0 ? p.cheb_hi : 1.2 * ws->lambda_max[pi];
    sl.lo = p.cheb_hi > 0 ? p.cheb_lo : sl.hi / 20.0;
  }
  // ||b||^2 (read by the host at the slot's first decision) and x = 0; nothing here waits for the GPU
  launch_dot(op, MFX_F64, op->n_dofs, b, b, ws->scal + 1, sl.stream);
  MFX_CUDA_TRY(cudaMemcpyAsync(sl.h_scal + 1, ws->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, sl.stream));
  MFX_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * op->n_dofs, sl.stream));
  sl.bb = 0.0;
  sl.bb_pending = true;
  rc = mixed ? capture_chunk<float>(sl, bt->chunk) : capture_chunk<double>(sl, bt->chunk);
  if (rc != MFX_OK) {
    slot_release(sl);
    return rc;
  }
  if (mixed) {
    sl.phase = SLOT_OUTER;
  } else {
    rc = slot_start_inner(sl);
    if (rc != MFX_OK) {
      slot_release(sl);
      return rc;
    }
    ws->h_st->done = 0;  // the first independent step launches the first chunk
  }
  *slot_out = free_slot;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

mfx_status mfx_batch_step(mfx_batch* bt, int32_t* n_active) {
  MFX_TRACE("mfx_batch_step");
  if (!bt) return set_error(MFX_EINVAL, "null batch");
  // 1) outer steps: residuals of the OUTER slots, then decide
  bool any_outer = false;
  for (auto& sl : bt->slots)
    if (sl.phase == SLOT_OUTER) {
      mfx_status rc = slot_launch_residual(sl);
      if (rc != MFX_OK) return rc;
      any_outer = true;
    }
  if (any_outer)
    for (auto& sl : bt->slots)
      if (sl.phase == SLOT_OUTER) MFX_CUDA_TRY(cudaStreamSynchronize(sl.stream));
  for (auto& sl : bt->slots) {
    if (sl.phase != SLOT_OUTER) continue;
    bool start = false;
    slot_outer_decide(sl, &start);
    if (start) {
      mfx_status rc = slot_start_inner(sl);
      if (rc != MFX_OK) return rc;
    }
  }
  // 2) one graph launch advances every INNER slot by a chunk of iterations
  mfx_status rc = rebuild_parent(bt);
  if (rc != MFX_OK) return rc;
  if (bt->parent) {
    for (int i : bt->parent_members)  // slot streams (inner starts) before the batch stream
      MFX_CUDA_TRY(cudaStreamSynchronize(bt->slots[i].stream));
    MFX_CUDA_TRY(cudaGraphLaunch(bt->parent, bt->stream));
    MFX_CUDA_TRY(cudaStreamSynchronize(bt->stream));
    ++bt->ticks;
  }
  // 3) finished inner solves
  int active = 0;
  for (auto& sl : bt->slots) {
    if (sl.phase == SLOT_INNER) {
      SolveWorkspace* ws = workspace(sl.op);
      const SolveState& h = *ws->h_st;
      if (h.done) {
        slot_read_bb(sl);
        sl.inner_total += h.it;
        if (h.status == MFX_BREAKDOWN) {
          sl.phase = SLOT_DONE;
          sl.status = MFX_BREAKDOWN;
        } else if (sl.mixed) {
          const int64_t n = sl.op->n_dofs;
          add_scaled_f32_kernel<<<vec_grid(n), 256, 0, sl.stream>>>(n, sl.x, ws->w32.x, ws->scal);
          sl.outer += 1;
          sl.phase = SLOT_OUTER;
        } else {
          MFX_CUDA_TRY(cudaMemcpyAsync(sl.x, ws->w64.x, sizeof(double) * sl.op->n_dofs, cudaMemcpyDeviceToDevice,
                                       sl.stream));
          sl.status = h.status;
          sl.phase = SLOT_DONE;
        }
      }
    }
    if (sl.phase == SLOT_OUTER || sl.phase == SLOT_INNER) ++active;
  }
  MFX_CUDA_TRY(cudaGetLastError());
  if (n_active) *n_active = active;
  return MFX_OK;
}

// Independent stepping: every slot whose previous work has finished takes its next step right
// away (residual, decision, inner start, next chunk), each on its own stream; nothing waits.
mfx_status mfx_batch_advance(mfx_batch* bt, int32_t* n_active) {
  MFX_TRACE("mfx_batch_advance");
  if (!bt) return set_error(MFX_EINVAL, "null batch");
  int active = 0;
  for (auto& sl : bt->slots) {
    if (sl.phase == SLOT_OUTER || sl.phase == SLOT_INNER) ++active;
    if (sl.phase != SLOT_OUTER && sl.phase != SLOT_INNER) continue;
    if (sl.busy) {
      const cudaError_t q = cudaEventQuery(sl.event);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return cuda_error(q, "mfx_batch_advance");
      sl.busy = false;
    }
    mfx_status rc = MFX_OK;
    if (sl.phase == SLOT_OUTER) {
      if (!sl.residual_pending) {
        rc = slot_launch_residual(sl);
        if (rc != MFX_OK) return rc;
        sl.residual_pending = true;
      } else {
        sl.residual_pending = false;
        bool start = false;
        slot_outer_decide(sl, &start);
        if (start) {
          rc = slot_start_inner(sl);
          if (rc != MFX_OK) return rc;
          MFX_CUDA_TRY(cudaGraphLaunch(sl.exec, sl.stream));
        }
      }
    } else {  // INNER: a chunk finished
      SolveWorkspace* ws = workspace(sl.op);
      const SolveState& h = *ws->h_st;
      if (!h.done) {
        MFX_CUDA_TRY(cudaGraphLaunch(sl.exec, sl.stream));
      } else {
        slot_read_bb(sl);
        sl.inner_total += h.it;
        if (h.status == MFX_BREAKDOWN) {
          sl.phase = SLOT_DONE;
          sl.status = MFX_BREAKDOWN;
        } else if (sl.mixed) {
          const int64_t n = sl.op->n_dofs;
          add_scaled_f32_kernel<<<vec_grid(n), 256, 0, sl.stream>>>(n, sl.x, ws->w32.x, ws->scal);
          sl.outer += 1;
          sl.phase = SLOT_OUTER;
          rc = slot_launch_residual(sl);
          if (rc != MFX_OK) return rc;
          sl.residual_pending = true;
        } else {
          MFX_CUDA_TRY(cudaMemcpyAsync(sl.x, ws->w64.x, sizeof(double) * sl.op->n_dofs, cudaMemcpyDeviceToDevice,
                                       sl.stream));
          sl.status = h.status;
          sl.phase = SLOT_DONE;
        }
      }
    }
    if (sl.phase == SLOT_OUTER || sl.phase == SLOT_INNER) {
      MFX_CUDA_TRY(cudaEventRecord(sl.event, sl.stream));
      sl.busy = true;
    } else {
      MFX_CUDA_TRY(cudaStreamSynchronize(sl.stream));  // results complete before the slot reports done
      --active;
    }
  }
  if (n_active) *n_active = active;
  return MFX_OK;
}

// Every active slot's whole solve (from x = 0) in one graph launch; the device decides when each
// problem stops (graph WHILE nodes whose conditions kernels set).
mfx_status mfx_batch_run(mfx_batch* bt, int32_t* n_done) try {
  MFX_TRACE("mfx_batch_run");
  if (!bt) return set_error(MFX_EINVAL, "null batch");
  std::vector<int> members;
  for (size_t i = 0; i < bt->slots.size(); ++i)
    if (bt->slots[i].phase == SLOT_OUTER || bt->slots[i].phase == SLOT_INNER) members.push_back((int)i);
  if (n_done) *n_done = 0;
  if (members.empty()) return MFX_OK;
  if (!bt->run_state) MFX_CUDA_TRY(cudaMalloc(&bt->run_state, sizeof(RunState) * bt->slots.size()));
  RunState* rs = reinterpret_cast<RunState*>(bt->run_state);
  for (int i : members) MFX_CUDA_TRY(cudaStreamSynchronize(bt->slots[i].stream));  // (b, b), x = 0 of the adds
  cudaGraph_t g = nullptr;
  MFX_CUDA_TRY(cudaGraphCreate(&g, 0));
  mfx_status rc = MFX_OK;
  for (int i : members) {
    BatchSlot& sl = bt->slots[i];
    rc = add_slot_solve(sl, bt->chunk, rs + i, g);
    if (rc != MFX_OK) break;
  }
  cudaGraphExec_t exec = nullptr;
  if (rc == MFX_OK) {
    cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) rc = cuda_error(e, "batch run: instantiate");
  }
  cudaGraphDestroy(g);
  if (rc != MFX_OK) return rc;
  cudaError_t e = cudaGraphLaunch(exec, bt->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(bt->stream);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return cuda_error(e, "batch run: launch");
  ++bt->runs;
  std::vector<RunState> h(bt->slots.size());
  MFX_CUDA_TRY(cudaMemcpy(h.data(), rs, sizeof(RunState) * h.size(), cudaMemcpyDeviceToHost));
  int done = 0;
  for (int i : members) {
    BatchSlot& sl = bt->slots[i];
    const RunState& r = h[i];
    sl.status = r.status;
    sl.bb = r.bb;
    sl.bb_pending = false;
    sl.rr = r.rr;
    sl.outer = sl.mixed ? r.outer : 0;
    sl.inner_total = r.inner_total;
    sl.phase = SLOT_DONE;
    ++done;
  }
  if (n_done) *n_done = done;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

mfx_status mfx_batch_poll(mfx_batch* bt, int32_t slot, int32_t* done, mfx_solve_stats* stats) {
  if (!bt || slot < 0 || slot >= (int)bt->slots.size() || !done) return set_error(MFX_EINVAL, "mfx_batch_poll");
  const BatchSlot& sl = bt->slots[slot];
  if (sl.phase == SLOT_FREE) return set_error(MFX_EINVAL, "slot is free");
  *done = sl.phase == SLOT_DONE ? 1 : 0;
  if (stats) {
    *stats = mfx_solve_stats{};
    stats->status = sl.status;
    stats->iterations = sl.mixed ? sl.outer : sl.inner_total;
    stats->inner_iterations = sl.mixed ? sl.inner_total : 0;
    stats->rel_residual = sl.bb > 0 ? std::sqrt(sl.rr / sl.bb) : 0.0;
    stats->cheb_lo = sl.lo;
    stats->cheb_hi = sl.hi;
  }
  return MFX_OK;
}

mfx_status mfx_batch_release(mfx_batch* bt, int32_t slot) {
  if (!bt || slot < 0 || slot >= (int)bt->slots.size()) return set_error(MFX_EINVAL, "mfx_batch_release");
  BatchSlot& sl = bt->slots[slot];
  if (sl.stream) MFX_CUDA_TRY(cudaStreamSynchronize(sl.stream));
  if (bt->parent) {
    // the parent graph holds a copy of this slot's chunk; rebuild it on the next step
    cudaGraphExecDestroy(bt->parent);
    bt->parent = nullptr;
    bt->parent_members.clear();
  }
  slot_release(sl);
  return MFX_OK;
}

}  // extern "C"

#include "mg.cuh"
