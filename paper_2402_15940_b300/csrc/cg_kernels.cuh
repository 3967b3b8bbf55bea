// Conjugate-gradient vector kernels with device-resident scalars (arXiv 2402.15940,
// Sec. 2.3: CG built from 1D vector kernels, the 3D operator kernel, warp-level dot
// products and a synchronisation mechanism).  Here each dot product is reduced with
// warp shuffles, then per block, then by the last block to finish (a ticket counter,
// no spinning), which also computes the CG scalars on the device.  The iteration loop
// itself runs inside a CUDA graph whose while-condition the last kernel sets, so the
// host never waits per iteration.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fepa {

struct CgState {
  double rho;       // (z, r)
  double alpha;     // rho / (d, h)
  double beta;      // rho_new / rho
  double bb;        // ||b||^2
  double rr;        // ||r||^2
  double tol2;      // rtol^2 ||b||^2
  int iter;         // iterations done
  int maxit;
  int done;         // set when converged or maxit reached
  int converged;
  unsigned int ticket;
  int tick_limit;   // the graph loop pauses (without finishing) once iter reaches this
};

// Resumable solves: allow `k` more iterations before the graph loop pauses.
__global__ void cg_set_tick(CgState* st, int k) {
  const long long lim = (long long)st->iter + k;
  st->tick_limit = lim > 0x7fffffff ? 0x7fffffff : (int)lim;
}

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NV values; thread 0 returns the sums in out[].
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (&out)[NV]) {
  __shared__ double red[NV][RED_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) red[k][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < RED_THREADS / 32; ++w) s += red[k][w];
      out[k] = s;
    }
  }
}

// Publish this block's partial sums; returns true (in thread 0) for the last block to
// arrive, after which partials[] of every block are visible to it.
template <int NV>
__device__ __forceinline__ bool publish_partials(double (&blk)[NV], double* partials, unsigned int* ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * gridDim.x + blockIdx.x] = blk[k];
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// Fixed-order final sum over block partials (deterministic for a fixed grid).
template <int NV>
__device__ __forceinline__ void final_sums(const double* partials, double (&out)[NV]) {
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    v[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v[k] += __ldcg(partials + k * gridDim.x + b);
  }
  block_sum<NV>(v, out);
}

// r = b - h; z = r * inv_diag (or r); d = z; h = 0; rho = (z,r), rr = (r,r), bb = (b,b)
__global__ void __launch_bounds__(RED_THREADS)
cg_init(int64_t N, const double* __restrict__ b, double* __restrict__ r, double* __restrict__ d,
        double* __restrict__ h, const double* __restrict__ inv_diag, CgState* st, double rtol2, int maxit,
        double* partials) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double ri = bi - h[i];
    const double zi = inv_diag ? ri * inv_diag[i] : ri;
    r[i] = ri;
    d[i] = zi;
    h[i] = 0.0;
    v[0] += zi * ri;
    v[1] += ri * ri;
    v[2] += bi * bi;
  }
  double blk[3];
  block_sum<3>(v, blk);
  if (publish_partials<3>(blk, partials, &st->ticket)) {
    double tot[3];
    final_sums<3>(partials, tot);
    if (threadIdx.x == 0) {
      st->rho = tot[0];
      st->rr = tot[1];
      st->bb = tot[2];
      st->tol2 = rtol2 * tot[2];
      st->iter = 0;
      st->maxit = maxit;
      st->converged = (tot[1] <= st->tol2 && isfinite(st->tol2)) ? 1 : 0;
      st->done = st->converged || !isfinite(st->rr) || !isfinite(st->bb);  // NaN/inf: stop at once
      st->alpha = st->beta = 0.0;
      st->tick_limit = 0x7fffffff;
      st->ticket = 0;
    }
  }
}

// alpha = rho / (d, h)
__global__ void __launch_bounds__(RED_THREADS)
cg_dot_dh(int64_t N, const double* __restrict__ d, const double* __restrict__ h, CgState* st, double* partials) {
  if (st->done) return;
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += d[i] * h[i];
  double blk[1];
  block_sum<1>(v, blk);
  if (publish_partials<1>(blk, partials, &st->ticket)) {
    double tot[1];
    final_sums<1>(partials, tot);
    if (threadIdx.x == 0) {
      st->alpha = st->rho / tot[0];
      st->ticket = 0;
    }
  }
}

// x += alpha d; r -= alpha h; rho_new = (z, r) with z = r * inv_diag; rr = (r, r);
// then the stopping test and beta.
__global__ void __launch_bounds__(RED_THREADS)
cg_update(int64_t N, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ d,
          const double* __restrict__ h, const double* __restrict__ inv_diag, CgState* st, double* partials) {
  if (st->done) return;
  const double alpha = st->alpha;
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * d[i];
    const double ri = r[i] - alpha * h[i];
    r[i] = ri;
    const double zi = inv_diag ? ri * inv_diag[i] : ri;
    v[0] += zi * ri;
    v[1] += ri * ri;
  }
  double blk[2];
  block_sum<2>(v, blk);
  if (publish_partials<2>(blk, partials, &st->ticket)) {
    double tot[2];
    final_sums<2>(partials, tot);
    if (threadIdx.x == 0) {
      st->iter += 1;
      st->rr = tot[1];
      if (tot[1] <= st->tol2) {
        st->converged = 1;
        st->done = 1;
      } else if (st->iter >= st->maxit || !isfinite(st->rr)) {
        st->done = 1;
      }
      st->beta = tot[0] / st->rho;
      st->rho = tot[0];
      st->ticket = 0;
    }
  }
}

// The FP64 loop's balanced pair (the graph and stream loops of fepa_cg_solve and the resumable
// solve): cg_update_r leaves x to cg_direction_x, which reads d anyway, so the update kernel makes
// four FP64 operations per DOF instead of five and moves 32 bytes instead of 56 -- B300's FP64
// pipe (about 0.6 T multiply-adds/s) and HBM bound cg_update about equally at large N.  The last
// step's x update is cg_flush64's.  Each value is computed as by cg_update / cg_direction (the same
// alpha, old d and operations), only one kernel later.
__global__ void __launch_bounds__(RED_THREADS)
cg_update_r(int64_t N, double* __restrict__ r, const double* __restrict__ h, const double* __restrict__ inv_diag,
            CgState* st, double* partials) {
  if (st->done) return;
  const double alpha = st->alpha;
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i] - alpha * h[i];
    r[i] = ri;
    const double zi = inv_diag ? ri * inv_diag[i] : ri;
    v[0] += zi * ri;
    v[1] += ri * ri;
  }
  double blk[2];
  block_sum<2>(v, blk);
  if (publish_partials<2>(blk, partials, &st->ticket)) {
    double tot[2];
    final_sums<2>(partials, tot);
    if (threadIdx.x == 0) {
      st->iter += 1;
      st->rr = tot[1];
      if (tot[1] <= st->tol2) {
        st->converged = 1;
        st->done = 1;
      } else if (st->iter >= st->maxit || !isfinite(st->rr)) {
        st->done = 1;
      }
      st->beta = tot[0] / st->rho;
      st->rho = tot[0];
      st->ticket = 0;
    }
  }
}

// x += alpha d (this iteration's step, d still the old direction); d = z + beta d; h = 0.  Block 0
// sets the graph's while-condition.  Once the loop is done nothing is written (cg_flush64).
__global__ void __launch_bounds__(RED_THREADS)
cg_direction_x(int64_t N, const double* __restrict__ r, double* __restrict__ d, double* __restrict__ h,
               const double* __restrict__ inv_diag, double* __restrict__ x, const CgState* st,
               cudaGraphConditionalHandle cond, int use_cond) {
  const int done = st->done;
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0)
    cudaGraphSetConditional(cond, (done || st->iter >= st->tick_limit) ? 0u : 1u);
  if (done) return;
  const double alpha = st->alpha, beta = st->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double di = d[i];
    x[i] += alpha * di;
    const double zi = inv_diag ? r[i] * inv_diag[i] : r[i];
    d[i] = zi + beta * di;
    h[i] = 0.0;
  }
}

// x += alpha d for the final step of a finished FP64 loop (done and at least one step): its
// direction kernel returned before advancing x
__global__ void cg_flush64(int64_t N, double* __restrict__ x, const double* __restrict__ d, const CgState* st) {
  if (!(st->done && st->iter > 0)) return;
  const double alpha = st->alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += alpha * d[i];
}

// d = z + beta d; h = 0.  Block 0 sets the graph's while-condition to !done.
__global__ void __launch_bounds__(RED_THREADS)
cg_direction(int64_t N, const double* __restrict__ r, double* __restrict__ d, double* __restrict__ h,
             const double* __restrict__ inv_diag, const CgState* st, cudaGraphConditionalHandle cond,
             int use_cond) {
  const int done = st->done;
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0)
    cudaGraphSetConditional(cond, (done || st->iter >= st->tick_limit) ? 0u : 1u);
  if (done) return;
  const double beta = st->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = inv_diag ? r[i] * inv_diag[i] : r[i];
    d[i] = zi + beta * d[i];
    h[i] = 0.0;
  }
}

__global__ void reciprocal(int64_t N, const double* __restrict__ a, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 1.0 / a[i];
}

__global__ void set_rows(int64_t count, const int* __restrict__ rows, double value, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    v[rows[i]] = value;
}

}  // namespace fepa

namespace fepa {

// ---------------------------------------------------------------------------
// Mixed precision: inner CG on FP32 vectors with the FP32 operator, inside FP64
// iterative refinement.  On this GPU the FP64 pipe is ~75x slower than FP32, so the
// inner loop keeps it idle: vector updates are FP32, and the dot products are
// accumulated per thread as an unevaluated sum of two floats (exact products by FMA,
// exact sums by TwoSum), i.e. to about 48 significant bits on the FP32 pipe, then
// combined across threads and blocks in FP64.  Scalars (alpha, beta, rho) stay FP64.
// ---------------------------------------------------------------------------
// Inner tolerance of a refinement step at outer residual rel: inner_rtol, relaxed when
// less is enough to reach rtol (the last correction: 0.25 rtol / rel, at most 0.5)
__host__ __device__ inline double inner_tol(double inner_rtol, double rtol, double rel) {
  const double need = rel > 0.0 ? 0.25 * rtol / rel : inner_rtol;
  return need > inner_rtol ? (need < 0.5 ? need : 0.5) : inner_rtol;
}

__device__ __forceinline__ void f2_add_prod(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);   // a*b - p exactly
  const float s = __fadd_rn(hi, p);
  const float bv = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));  // hi + p - s exactly
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ double f2_value(float hi, float lo) { return (double)hi + (double)lo; }

// x = 0; r = b; z = r * inv_diag; d = z; h = 0; rho = (z,r), rr = (r,r), bb = (b,b)
__global__ void __launch_bounds__(RED_THREADS)
cg32_init(int64_t N, const float* __restrict__ b, float* __restrict__ x, float* __restrict__ r,
          float* __restrict__ d, float* __restrict__ h, const float* __restrict__ inv_diag, CgState* st,
          double rtol2, int maxit, double* partials) {
  float zr_h = 0.f, zr_l = 0.f, rr_h = 0.f, rr_l = 0.f, bb_h = 0.f, bb_l = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float ri = b[i];
    const float zi = inv_diag ? ri * inv_diag[i] : ri;
    x[i] = 0.f;
    r[i] = ri;
    d[i] = zi;
    h[i] = 0.f;
    f2_add_prod(zr_h, zr_l, zi, ri);
    f2_add_prod(rr_h, rr_l, ri, ri);
    f2_add_prod(bb_h, bb_l, ri, ri);
  }
  double v[3] = {f2_value(zr_h, zr_l), f2_value(rr_h, rr_l), f2_value(bb_h, bb_l)};
  double blk[3];
  block_sum<3>(v, blk);
  if (publish_partials<3>(blk, partials, &st->ticket)) {
    double tot[3];
    final_sums<3>(partials, tot);
    if (threadIdx.x == 0) {
      st->rho = tot[0];
      st->rr = tot[1];
      st->bb = tot[2];
      st->tol2 = rtol2 * tot[2];
      st->iter = 0;
      st->maxit = maxit;
      st->converged = (tot[1] <= st->tol2 && isfinite(st->tol2)) ? 1 : 0;
      st->done = st->converged || !isfinite(st->rr) || !isfinite(st->bb);  // NaN/inf: stop at once
      st->alpha = st->beta = 0.0;
      st->tick_limit = 0x7fffffff;
      st->ticket = 0;
    }
  }
}

__global__ void __launch_bounds__(RED_THREADS)
cg32_dot_dh(int64_t N, const float* __restrict__ d, const float* __restrict__ h, CgState* st, double* partials) {
  if (st->done) return;
  float s_h = 0.f, s_l = 0.f;
  // 16-byte vector loads over the bulk (the loop's vectors are 256-byte aligned), scalar tail
  const int64_t N4 = N >> 2, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, ts = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = t0; i < N4; i += ts) {
    const float4 dv = reinterpret_cast<const float4*>(d)[i], hv = reinterpret_cast<const float4*>(h)[i];
    f2_add_prod(s_h, s_l, dv.x, hv.x);
    f2_add_prod(s_h, s_l, dv.y, hv.y);
    f2_add_prod(s_h, s_l, dv.z, hv.z);
    f2_add_prod(s_h, s_l, dv.w, hv.w);
  }
  for (int64_t i = 4 * N4 + t0; i < N; i += ts) f2_add_prod(s_h, s_l, d[i], h[i]);
  double v[1] = {f2_value(s_h, s_l)};
  double blk[1];
  block_sum<1>(v, blk);
  if (publish_partials<1>(blk, partials, &st->ticket)) {
    double tot[1];
    final_sums<1>(partials, tot);
    if (threadIdx.x == 0) {
      st->alpha = st->rho / tot[0];
      st->ticket = 0;
    }
  }
}

// r -= alpha h; rho_new = (z, r) with z = r * inv_diag; rr = (r, r); stop test.  (x is
// advanced by the direction kernel, which reads d anyway: one N-vector pass fewer per
// iteration; the last iteration's x update is applied by cg32_flush.)  dh_slots: the
// action kernel accumulated (d, h) into these RED_THREADS doubles; every block sums them
// and forms alpha = rho / (d, h) itself (block 0 also stores it); null: alpha is st->alpha.
__global__ void __launch_bounds__(RED_THREADS)
cg32_update(int64_t N, float* __restrict__ r, const float* __restrict__ h, const float* __restrict__ inv_diag,
            CgState* st, double* partials, const double* __restrict__ dh_slots) {
  if (st->done) return;
  float alpha;
  if (dh_slots) {
    __shared__ double s_alpha;
    double v[1] = {__ldcg(dh_slots + threadIdx.x)}, tot[1];
    block_sum<1>(v, tot);
    if (threadIdx.x == 0) {
      s_alpha = st->rho / tot[0];
      if (blockIdx.x == 0) st->alpha = s_alpha;
    }
    __syncthreads();
    alpha = (float)s_alpha;
  } else {
    alpha = (float)st->alpha;
  }
  float zr_h = 0.f, zr_l = 0.f, rr_h = 0.f, rr_l = 0.f;
  auto one = [&](float& ri, float hi, float wi) {
    ri = fmaf(-alpha, hi, ri);
    f2_add_prod(zr_h, zr_l, ri * wi, ri);
    f2_add_prod(rr_h, rr_l, ri, ri);
  };
  const int64_t N4 = N >> 2, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, ts = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = t0; i < N4; i += ts) {  // 16-byte vector accesses over the bulk
    float4 rv = reinterpret_cast<float4*>(r)[i];
    const float4 hv = reinterpret_cast<const float4*>(h)[i];
    const float4 wv = inv_diag ? reinterpret_cast<const float4*>(inv_diag)[i] : make_float4(1.f, 1.f, 1.f, 1.f);
    one(rv.x, hv.x, wv.x);
    one(rv.y, hv.y, wv.y);
    one(rv.z, hv.z, wv.z);
    one(rv.w, hv.w, wv.w);
    reinterpret_cast<float4*>(r)[i] = rv;
  }
  for (int64_t i = 4 * N4 + t0; i < N; i += ts) one(r[i], h[i], inv_diag ? inv_diag[i] : 1.f);
  double v[2] = {f2_value(zr_h, zr_l), f2_value(rr_h, rr_l)};
  double blk[2];
  block_sum<2>(v, blk);
  if (publish_partials<2>(blk, partials, &st->ticket)) {
    double tot[2];
    final_sums<2>(partials, tot);
    if (threadIdx.x == 0) {
      st->iter += 1;
      st->rr = tot[1];
      if (tot[1] <= st->tol2) {
        st->converged = 1;
        st->done = 1;
      } else if (st->iter >= st->maxit || !isfinite(st->rr)) {
        st->done = 1;
      }
      st->beta = tot[0] / st->rho;
      st->rho = tot[0];
      st->ticket = 0;
    }
  }
}

// With update_x: x += alpha d (this iteration's step, d still the old direction); then
// d = z + beta d and h = 0 for the next action.  Block 0 sets the while-condition and
// clears dh_slots (if given) for the next action's (d, h).  Once the loop is done nothing
// else is written: the final step's x update is cg32_flush's.
__global__ void __launch_bounds__(RED_THREADS)
cg32_direction(int64_t N, const float* __restrict__ r, float* __restrict__ d, float* __restrict__ h,
               const float* __restrict__ inv_diag, float* __restrict__ x, int update_x, const CgState* st,
               cudaGraphConditionalHandle cond, int use_cond, double* __restrict__ dh_slots) {
  if (dh_slots && blockIdx.x == 0) dh_slots[threadIdx.x] = 0.0;
  const int done = st->done;
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0)
    cudaGraphSetConditional(cond, (done || st->iter >= st->tick_limit) ? 0u : 1u);
  if (done) return;
  const float beta = (float)st->beta, alpha = update_x ? (float)st->alpha : 0.f;
  const int64_t N4 = N >> 2, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, ts = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = t0; i < N4; i += ts) {  // 16-byte vector accesses over the bulk
    const float4 rv = reinterpret_cast<const float4*>(r)[i];
    const float4 wv = inv_diag ? reinterpret_cast<const float4*>(inv_diag)[i] : make_float4(1.f, 1.f, 1.f, 1.f);
    float4 dv = reinterpret_cast<float4*>(d)[i];
    if (update_x) {
      float4 xv = reinterpret_cast<float4*>(x)[i];
      xv.x = fmaf(alpha, dv.x, xv.x);
      xv.y = fmaf(alpha, dv.y, xv.y);
      xv.z = fmaf(alpha, dv.z, xv.z);
      xv.w = fmaf(alpha, dv.w, xv.w);
      reinterpret_cast<float4*>(x)[i] = xv;
    }
    dv.x = fmaf(beta, dv.x, rv.x * wv.x);
    dv.y = fmaf(beta, dv.y, rv.y * wv.y);
    dv.z = fmaf(beta, dv.z, rv.z * wv.z);
    dv.w = fmaf(beta, dv.w, rv.w * wv.w);
    reinterpret_cast<float4*>(d)[i] = dv;
    reinterpret_cast<float4*>(h)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int64_t i = 4 * N4 + t0; i < N; i += ts) {
    if (update_x) x[i] = fmaf(alpha, d[i], x[i]);
    const float zi = inv_diag ? r[i] * inv_diag[i] : r[i];
    d[i] = fmaf(beta, d[i], zi);
    h[i] = 0.f;
  }
}

// (x, y) of two FP32 vectors added into the DOT_SLOTS-style slots (RED_THREADS doubles,
// slot blockIdx.x mod RED_THREADS): the unfused form of the action kernel's (x, A x)
__global__ void __launch_bounds__(RED_THREADS)
dot32_slots(int64_t N, const float* __restrict__ x, const float* __restrict__ y, double* slots) {
  float s_h = 0.f, s_l = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    f2_add_prod(s_h, s_l, x[i], y[i]);
  double v[1] = {f2_value(s_h, s_l)}, blk[1];
  block_sum<1>(v, blk);
  if (threadIdx.x == 0) atomicAdd(slots + blockIdx.x % RED_THREADS, blk[0]);
}

// *out = sum of the RED_THREADS slots, which are cleared for the next use (one block)
__global__ void __launch_bounds__(RED_THREADS) dot_collect(double* slots, double* out) {
  double v[1] = {slots[threadIdx.x]}, tot[1];
  slots[threadIdx.x] = 0.0;
  block_sum<1>(v, tot);
  if (threadIdx.x == 0) *out = tot[0];
}

// x += alpha d for the final step of a finished FP32 loop (done and at least one step):
// its direction kernel returned before advancing x
__global__ void cg32_flush(int64_t N, float* __restrict__ x, const float* __restrict__ d, const CgState* st) {
  if (!(st->done && st->iter > 0)) return;
  const float alpha = (float)st->alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fmaf(alpha, d[i], x[i]);
}

// Outer step of the refinement: r = b - h in FP64 (h = A x from the FP64 operator),
// handed to the inner solve as r32; ||r||^2 and ||b||^2 in FP64 into st->rr, st->bb.
__global__ void __launch_bounds__(RED_THREADS)
refine_residual(int64_t N, const double* __restrict__ b, const double* __restrict__ h, float* __restrict__ r32,
                CgState* st, double* partials) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double ri = bi - h[i];
    r32[i] = (float)ri;
    v[0] += ri * ri;
    v[1] += bi * bi;
  }
  double blk[2];
  block_sum<2>(v, blk);
  if (publish_partials<2>(blk, partials, &st->ticket)) {
    double tot[2];
    final_sums<2>(partials, tot);
    if (threadIdx.x == 0) {
      st->rr = tot[0];
      st->bb = tot[1];
      st->ticket = 0;
    }
  }
}

// Residual replacement for the reliable-update solve: the FP32 loop stopped after its
// residual fell by delta; x has absorbed e, r holds the FP64 residual b - A x rounded to
// FP32.  Here: e = 0; rho = (z, r), rr = (r, r) of the replaced residual; beta so that
// the following direction kernel gives d = z + (rho / rho_prev) d_prev, continuing the
// same Krylov recurrence (rho_prev = rho_last / beta_last); stop the next segment at
// rr <= max(delta2 rr, floor2).
__global__ void __launch_bounds__(RED_THREADS)
cg32_replace(int64_t N, const float* __restrict__ r, float* __restrict__ e, const float* __restrict__ inv_diag,
             CgState* st, double delta2, double floor2, double* partials) {
  float zr_h = 0.f, zr_l = 0.f, rr_h = 0.f, rr_l = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float ri = r[i];
    const float zi = inv_diag ? ri * inv_diag[i] : ri;
    e[i] = 0.f;
    f2_add_prod(zr_h, zr_l, zi, ri);
    f2_add_prod(rr_h, rr_l, ri, ri);
  }
  double v[2] = {f2_value(zr_h, zr_l), f2_value(rr_h, rr_l)};
  double blk[2];
  block_sum<2>(v, blk);
  if (publish_partials<2>(blk, partials, &st->ticket)) {
    double tot[2];
    final_sums<2>(partials, tot);
    if (threadIdx.x == 0) {
      // (no step taken since the last start: beta 0 restarts the direction at d = z)
      st->beta = st->beta != 0.0 ? tot[0] / (st->rho / st->beta) : 0.0;
      st->rho = tot[0];
      st->rr = tot[1];
      st->tol2 = delta2 * tot[1] > floor2 ? delta2 * tot[1] : floor2;
      st->converged = 0;
      st->done = 0;
      st->ticket = 0;
    }
  }
}

// x += e (FP64 accumulation of the FP32 correction)
// x += escale e (escale: the power of two the residual was scaled down by, or 1)
__global__ void refine_correct(int64_t N, double* __restrict__ x, const float* __restrict__ e, double escale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += escale * (double)e[i];
}

// The residual handed to the FP32 inner solve again, r32 = (b - h) rscale, when its norm is so
// small or large that FP32 products of it would leave the float range (rscale: a power of two)
__global__ void refine_rescale(int64_t N, const double* __restrict__ b, const double* __restrict__ h,
                               float* __restrict__ r32, double rscale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    r32[i] = (float)((b[i] - h[i]) * rscale);
}

__global__ void to_f32(int64_t N, const double* __restrict__ a, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)a[i];
}

}  // namespace fepa
