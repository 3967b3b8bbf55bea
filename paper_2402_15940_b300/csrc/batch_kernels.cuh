// Batched Jacobi-PCG over many independent problems at once (one concatenated vector,
// per-problem scalars).  The DOFs are cut into chunks of one problem each (the chunk table
// below); every reduction writes one partial per chunk and the last block to finish sums each
// problem's chunk partials in a fixed order and updates that problem's scalars, so a problem's
// iterates do not depend on which other problems share the batch (up to the atomic order of
// G^T).  The kernels are persistent: a fixed grid walks its chunks (or, inside the iteration
// loop, only the chunks of problems still running, from a work list), so finished problems
// cost no block launches; the loop runs inside one CUDA graph while-node until the last
// problem stops.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_kernels.cuh"

namespace fepa {

struct BState {  // per problem
  double rho, alpha, beta, bb, rr, tol2;
  int iter, maxit, converged, pad;
};

struct BGlobal {  // whole batch
  unsigned int ticket;
  int active;  // problems still iterating
  int done;    // 1 when none is
  int pad;
};

struct ChunkTable {
  const int* blk_prob;     // [nchunks] problem of each chunk
  const int64_t* blk_lo;   // [nchunks] first DOF (concatenated numbering)
  const int64_t* blk_hi;   // [nchunks] one past the last DOF
  const int* pb_first;     // [nprob] first chunk of each problem
  const int* pb_count;     // [nprob] chunks of each problem
  int nprob;
  int nchunks;
  const int* act;          // the chunks of running problems (work list; null: every chunk)
  const int* nact;         // its length
  const int* aprob;        // the running problems (work list; null: every problem)
  const int* naprob;       // its length
};

// Work lists of the iteration loop, rebuilt whenever the set of running problems changes: the
// chunks of running problems, and per group the element tiles (of one problem each) of running
// problems, for the persistent operator kernels
struct WorkLists {
  int* act_chunks;          // [nchunks]
  int* n_act_chunks;        // [1]
  int* act_probs;           // [nprob]
  int* n_act_probs;         // [1]
  int ngroups;
  const int* prob_group;    // [nprob] group of each problem
  const int* tile_first;    // [nprob] first tile of the problem in its group's tile table
  const int* tile_count;    // [nprob] its tiles
  const int* tile_off;      // [ngroups] start of group g's list in act_tiles
  int* act_tiles;           // per group: tile ids of running problems
  int* n_act_tiles;         // [ngroups]
};

__device__ __forceinline__ int chunk_count(const ChunkTable& t) { return t.act ? *t.nact : t.nchunks; }
__device__ __forceinline__ int chunk_at(const ChunkTable& t, int i) { return t.act ? t.act[i] : i; }

// Block-reduce this block's NV values over one chunk and store them as the chunk's partials
template <int NV>
__device__ __forceinline__ void store_chunk(double (&v)[NV], double* partials, int nchunks, int chunk) {
  double blk[NV];
  block_sum<NV>(v, blk);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * nchunks + chunk] = blk[k];
  }
  __syncthreads();  // (block_sum's shared slots are reused by the next chunk)
}

// True (in every thread) in the last block to finish; every chunk partial is then visible to it
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  return last;
}

// Sum, per problem, the NV chunk partials of its chunks (called by the last block): one warp
// per problem, its lanes striding over the chunks and a fixed shuffle tree combining them (the
// order depends only on the problem's own chunk count); over every problem, or over the work
// list of running problems where the table carries one.  f(j, sums) -- called by one lane --
// receives problem j's totals.  Returns the number of problems f reports as active, summed over
// the block (valid in every thread after the call).
template <int NV, typename F>
__device__ __forceinline__ int per_problem(const ChunkTable& t, const double* partials, F f) {
  __shared__ int active;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int np = t.aprob ? *t.naprob : t.nprob;
  int mine = 0;
  for (int jj = threadIdx.x >> 5; jj < np; jj += nw) {
    const int j = t.aprob ? t.aprob[jj] : jj;
    const int b0 = t.pb_first[j], b1 = b0 + t.pb_count[j];
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      s[k] = 0.0;
      for (int b = b0 + lane; b < b1; b += 32) s[k] += __ldcg(partials + k * t.nchunks + b);
      s[k] = warp_sum(s[k]);
    }
    if (lane == 0) mine += f(j, s) ? 1 : 0;
  }
  atomicAdd(&active, mine);
  __syncthreads();
  return active;
}

// Rebuild the work lists from pdone (called by one whole block; w.act_chunks null: no lists)
__device__ __forceinline__ void rebuild_lists(const ChunkTable& t, const WorkLists& w, const int* pdone) {
  if (!w.act_chunks) return;
  if (threadIdx.x == 0) {
    *w.n_act_chunks = 0;
    *w.n_act_probs = 0;
  }
  for (int g = threadIdx.x; g < w.ngroups; g += blockDim.x) w.n_act_tiles[g] = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < t.nprob; j += blockDim.x) {
    if (__ldcg(pdone + j)) continue;
    w.act_probs[atomicAdd(w.n_act_probs, 1)] = j;
    const int nc = t.pb_count[j];
    const int cb = atomicAdd(w.n_act_chunks, nc);
    for (int c = 0; c < nc; ++c) w.act_chunks[cb + c] = t.pb_first[j] + c;
    const int g = w.prob_group[j], nt = w.tile_count[j];
    int* dst = w.act_tiles + w.tile_off[g] + atomicAdd(w.n_act_tiles + g, nt);
    for (int k = 0; k < nt; ++k) dst[k] = w.tile_first[j] + k;
  }
  __threadfence();
  __syncthreads();
}

__global__ void __launch_bounds__(RED_THREADS)
bcg_init(ChunkTable t, WorkLists w, const double* __restrict__ b, double* __restrict__ r, double* __restrict__ d,
         double* __restrict__ h, const double* __restrict__ inv_diag, BState* ps, int* pdone, BGlobal* gs,
         double rtol2, int maxit, double* partials) {
  for (int ic = blockIdx.x; ic < t.nchunks; ic += gridDim.x) {
    const int64_t lo = t.blk_lo[ic], hi = t.blk_hi[ic];
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
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
    store_chunk<3>(v, partials, t.nchunks, ic);
  }
  if (last_block(&gs->ticket)) {
    const int active = per_problem<3>(t, partials, [&](int j, const double* s) {
      BState& q = ps[j];
      q.rho = s[0];
      q.rr = s[1];
      q.bb = s[2];
      q.tol2 = rtol2 * s[2];
      q.iter = 0;
      q.maxit = maxit;
      q.alpha = q.beta = 0.0;
      q.converged = (s[1] <= q.tol2 && isfinite(q.tol2)) ? 1 : 0;
      pdone[j] = q.converged || !isfinite(s[1]) || !isfinite(s[2]);  // NaN/inf: stop at once
      return !pdone[j];
    });
    rebuild_lists(t, w, pdone);
    if (threadIdx.x == 0) {
      gs->active = active;
      gs->done = active == 0;
      gs->ticket = 0;
    }
  }
}

__global__ void __launch_bounds__(RED_THREADS)
bcg_dot_dh(ChunkTable t, const double* __restrict__ d, const double* __restrict__ h, BState* ps,
           const int* __restrict__ pdone, BGlobal* gs, double* partials) {
  if (gs->done) return;
  const int nc = chunk_count(t);
  for (int ic = blockIdx.x; ic < nc; ic += gridDim.x) {
    const int c = chunk_at(t, ic);
    double v[1] = {0.0};
    if (!pdone[t.blk_prob[c]]) {
      const int64_t lo = t.blk_lo[c], hi = t.blk_hi[c];
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) v[0] += d[i] * h[i];
    }
    store_chunk<1>(v, partials, t.nchunks, c);
  }
  if (last_block(&gs->ticket)) {
    per_problem<1>(t, partials, [&](int j, const double* s) {
      if (!pdone[j]) ps[j].alpha = ps[j].rho / s[0];
      return false;
    });
    if (threadIdx.x == 0) gs->ticket = 0;
  }
}

__global__ void __launch_bounds__(RED_THREADS)
bcg_update(ChunkTable t, WorkLists w, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ d,
           const double* __restrict__ h, const double* __restrict__ inv_diag, BState* ps, int* pdone, BGlobal* gs,
           double* partials) {
  if (gs->done) return;
  const int nc = chunk_count(t);
  for (int ic = blockIdx.x; ic < nc; ic += gridDim.x) {
    const int c = chunk_at(t, ic);
    const int prob = t.blk_prob[c];
    double v[2] = {0.0, 0.0};
    if (!pdone[prob]) {
      const double alpha = ps[prob].alpha;
      const int64_t lo = t.blk_lo[c], hi = t.blk_hi[c];
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        x[i] += alpha * d[i];
        const double ri = r[i] - alpha * h[i];
        r[i] = ri;
        const double zi = inv_diag ? ri * inv_diag[i] : ri;
        v[0] += zi * ri;
        v[1] += ri * ri;
      }
    }
    store_chunk<2>(v, partials, t.nchunks, c);
  }
  if (last_block(&gs->ticket)) {
    __shared__ int stopped;
    if (threadIdx.x == 0) stopped = 0;
    __syncthreads();
    const int active = per_problem<2>(t, partials, [&](int j, const double* s) {
      if (pdone[j]) return false;
      BState& q = ps[j];
      q.iter += 1;
      q.rr = s[1];
      int stop = 0;
      if (s[1] <= q.tol2) {
        q.converged = 1;
        stop = 1;
      } else if (q.iter >= q.maxit || !isfinite(q.rr)) {
        stop = 1;
      }
      q.beta = s[0] / q.rho;
      q.rho = s[0];
      pdone[j] = stop;
      if (stop) stopped = 1;
      return !stop;
    });
    if (stopped) rebuild_lists(t, w, pdone);  // (block-uniform after per_problem's barrier)
    if (threadIdx.x == 0) {
      gs->active = active;
      gs->done = active == 0;
      gs->ticket = 0;
    }
  }
}

// d = z + beta d, h = 0 for problems still iterating; block 0 sets the while-condition
__global__ void __launch_bounds__(RED_THREADS)
bcg_direction(ChunkTable t, const double* __restrict__ r, double* __restrict__ d, double* __restrict__ h,
              const double* __restrict__ inv_diag, const BState* ps, const int* __restrict__ pdone,
              const BGlobal* gs, cudaGraphConditionalHandle cond, int use_cond) {
  const int done = gs->done;
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, done ? 0u : 1u);
  if (done) return;
  const int nc = chunk_count(t);
  for (int ic = blockIdx.x; ic < nc; ic += gridDim.x) {
    const int c = chunk_at(t, ic);
    const int prob = t.blk_prob[c];
    if (pdone[prob]) continue;
    const double beta = ps[prob].beta;
    const int64_t lo = t.blk_lo[c], hi = t.blk_hi[c];
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const double zi = inv_diag ? r[i] * inv_diag[i] : r[i];
      d[i] = zi + beta * d[i];
      h[i] = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// Batched mixed-precision refinement: per problem, FP64 residual -> FP32 Jacobi-PCG
// correction (per-problem stop) -> FP64 update, as the single-problem refinement.  The
// FP32 kernels mirror the FP64 ones above with FP32 vectors and two-float dot products.
// ---------------------------------------------------------------------------

// r32 = b - h rounded to FP32 (h = A x from the FP64 action); per problem rr = ||r||^2,
// bb = ||b||^2 into pr; a problem whose rr <= rtol2 bb is finished (pdone = 1).
__global__ void __launch_bounds__(RED_THREADS)
bref_residual(ChunkTable t, const double* __restrict__ b, const double* __restrict__ h, float* __restrict__ r32,
              BState* pr, int* pdone, BGlobal* gs, double rtol2, double* partials) {
  for (int ic = blockIdx.x; ic < t.nchunks; ic += gridDim.x) {
    const int64_t lo = t.blk_lo[ic], hi = t.blk_hi[ic];
    double v[2] = {0.0, 0.0};
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const double bi = b[i];
      const double ri = bi - h[i];
      r32[i] = (float)ri;
      v[0] += ri * ri;
      v[1] += bi * bi;
    }
    store_chunk<2>(v, partials, t.nchunks, ic);
  }
  if (last_block(&gs->ticket)) {
    const int active = per_problem<2>(t, partials, [&](int j, const double* s) {
      BState& q = pr[j];
      q.rr = s[0];
      q.bb = s[1];
      q.converged = s[0] <= rtol2 * s[1] ? 1 : 0;
      pdone[j] = q.converged;
      return !q.converged;
    });
    if (threadIdx.x == 0) {
      gs->active = active;
      gs->done = active == 0;
      gs->ticket = 0;
    }
  }
}

// Start of the FP32 correction solves A e = r: e = 0, d = z, h = 0 everywhere; for every
// problem not finished, rho = (z, r), rr = (r, r) and the stop at rr <= tol^2 ||r||^2 with
// tol = inner_tol(inner_rtol, rtol, its outer residual) -- or, for the reliable-update solve
// (delta2 > 0), the first segment's stop at rr <= max(delta2 ||r||^2, rtol^2 ||b||^2 / 4).
__global__ void __launch_bounds__(RED_THREADS)
bcg32_init(ChunkTable t, WorkLists w, const float* __restrict__ r, float* __restrict__ e, float* __restrict__ d,
           float* __restrict__ h, const float* __restrict__ inv_diag, BState* ps, const BState* __restrict__ pr,
           int* pdone, BGlobal* gs, double inner_rtol, double rtol, int maxit, double delta2, double* partials) {
  for (int ic = blockIdx.x; ic < t.nchunks; ic += gridDim.x) {
    const int64_t lo = t.blk_lo[ic], hi = t.blk_hi[ic];
    float zr_h = 0.f, zr_l = 0.f, rr_h = 0.f, rr_l = 0.f;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const float ri = r[i];
      const float zi = inv_diag ? ri * inv_diag[i] : ri;
      e[i] = 0.f;
      d[i] = zi;
      h[i] = 0.f;
      f2_add_prod(zr_h, zr_l, zi, ri);
      f2_add_prod(rr_h, rr_l, ri, ri);
    }
    double v[2] = {f2_value(zr_h, zr_l), f2_value(rr_h, rr_l)};
    store_chunk<2>(v, partials, t.nchunks, ic);
  }
  if (last_block(&gs->ticket)) {
    const int active = per_problem<2>(t, partials, [&](int j, const double* s) {
      BState& q = ps[j];
      q.iter = 0;
      q.maxit = maxit;
      q.alpha = q.beta = 0.0;
      q.rho = s[0];
      q.rr = s[1];
      q.bb = s[1];
      if (pdone[j]) {  // finished by the outer test: no correction
        q.converged = 1;
        q.tol2 = 0.0;
        return false;
      }
      if (delta2 > 0.0) {
        const double floor2 = 0.25 * rtol * rtol * pr[j].bb;
        q.tol2 = delta2 * s[1] > floor2 ? delta2 * s[1] : floor2;
      } else {
        const double rel = pr[j].bb > 0.0 ? sqrt(pr[j].rr / pr[j].bb) : 0.0;
        const double tol = inner_tol(inner_rtol, rtol, rel);
        q.tol2 = tol * tol * s[1];
      }
      q.converged = s[1] <= q.tol2 ? 1 : 0;
      pdone[j] = q.converged;
      return !q.converged;
    });
    rebuild_lists(t, w, pdone);
    if (threadIdx.x == 0) {
      gs->active = active;
      gs->done = active == 0;
      gs->ticket = 0;
    }
  }
}

__global__ void __launch_bounds__(RED_THREADS)
bcg32_dot_dh(ChunkTable t, const float* __restrict__ d, const float* __restrict__ h, BState* ps,
             const int* __restrict__ pdone, BGlobal* gs, double* partials) {
  if (gs->done) return;
  const int nc = chunk_count(t);
  for (int ic = blockIdx.x; ic < nc; ic += gridDim.x) {
    const int c = chunk_at(t, ic);
    float s_h = 0.f, s_l = 0.f;
    if (!pdone[t.blk_prob[c]]) {
      const int64_t lo = t.blk_lo[c], hi = t.blk_hi[c];
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) f2_add_prod(s_h, s_l, d[i], h[i]);
    }
    double v[1] = {f2_value(s_h, s_l)};
    store_chunk<1>(v, partials, t.nchunks, c);
  }
  if (last_block(&gs->ticket)) {
    per_problem<1>(t, partials, [&](int j, const double* s) {
      if (!pdone[j]) ps[j].alpha = ps[j].rho / s[0];
      return false;
    });
    if (threadIdx.x == 0) gs->ticket = 0;
  }
}

__global__ void __launch_bounds__(RED_THREADS)
bcg32_update(ChunkTable t, WorkLists w, float* __restrict__ e, float* __restrict__ r, const float* __restrict__ d,
             const float* __restrict__ h, const float* __restrict__ inv_diag, BState* ps, int* pdone, BGlobal* gs,
             double* partials) {
  if (gs->done) return;
  const int nc = chunk_count(t);
  for (int ic = blockIdx.x; ic < nc; ic += gridDim.x) {
    const int c = chunk_at(t, ic);
    const int prob = t.blk_prob[c];
    float zr_h = 0.f, zr_l = 0.f, rr_h = 0.f, rr_l = 0.f;
    if (!pdone[prob]) {
      const float alpha = (float)ps[prob].alpha;
      const int64_t lo = t.blk_lo[c], hi = t.blk_hi[c];
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        e[i] = fmaf(alpha, d[i], e[i]);
        const float ri = fmaf(-alpha, h[i], r[i]);
        r[i] = ri;
        const float zi = inv_diag ? ri * inv_diag[i] : ri;
        f2_add_prod(zr_h, zr_l, zi, ri);
        f2_add_prod(rr_h, rr_l, ri, ri);
      }
    }
    double v[2] = {f2_value(zr_h, zr_l), f2_value(rr_h, rr_l)};
    store_chunk<2>(v, partials, t.nchunks, c);
  }
  if (last_block(&gs->ticket)) {
    __shared__ int stopped;
    if (threadIdx.x == 0) stopped = 0;
    __syncthreads();
    const int active = per_problem<2>(t, partials, [&](int j, const double* s) {
      if (pdone[j]) return false;
      BState& q = ps[j];
      q.iter += 1;
      q.rr = s[1];
      int stop = 0;
      if (s[1] <= q.tol2) {
        q.converged = 1;
        stop = 1;
      } else if (q.iter >= q.maxit || !isfinite(q.rr)) {
        stop = 1;
      }
      q.beta = s[0] / q.rho;
      q.rho = s[0];
      pdone[j] = stop;
      if (stop) stopped = 1;
      return !stop;
    });
    if (stopped) rebuild_lists(t, w, pdone);  // (block-uniform after per_problem's barrier)
    if (threadIdx.x == 0) {
      gs->active = active;
      gs->done = active == 0;
      gs->ticket = 0;
    }
  }
}

// Residual replacement of the batched reliable-update solve (as cg32_replace, per problem):
// r holds each problem's FP64 residual b - A x rounded to FP32 and e = 0; every problem not
// finished by the FP64 test (pdone 0) and below maxit gets rho = (z, r), rr = (r, r), beta
// rescaled so that the next direction continues its recurrence (d = z + rho / rho_prev d),
// and its next stop at rr <= max(delta2 rr, rtol^2 ||b||^2 / 4); the others stop.
__global__ void __launch_bounds__(RED_THREADS)
bcg32_replace(ChunkTable t, WorkLists w, const float* __restrict__ r, float* __restrict__ e,
              const float* __restrict__ inv_diag, BState* ps, const BState* __restrict__ pr, int* pdone, BGlobal* gs,
              double delta2, double rtol, double* partials) {
  for (int ic = blockIdx.x; ic < t.nchunks; ic += gridDim.x) {
    const int64_t lo = t.blk_lo[ic], hi = t.blk_hi[ic];
    float zr_h = 0.f, zr_l = 0.f, rr_h = 0.f, rr_l = 0.f;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const float ri = r[i];
      const float zi = inv_diag ? ri * inv_diag[i] : ri;
      e[i] = 0.f;
      f2_add_prod(zr_h, zr_l, zi, ri);
      f2_add_prod(rr_h, rr_l, ri, ri);
    }
    double v[2] = {f2_value(zr_h, zr_l), f2_value(rr_h, rr_l)};
    store_chunk<2>(v, partials, t.nchunks, ic);
  }
  if (last_block(&gs->ticket)) {
    const int active = per_problem<2>(t, partials, [&](int j, const double* s) {
      BState& q = ps[j];
      if (pdone[j] || q.iter >= q.maxit) {
        pdone[j] = 1;
        return false;
      }
      q.beta = q.beta != 0.0 ? s[0] / (q.rho / q.beta) : 0.0;
      q.rho = s[0];
      q.rr = s[1];
      const double floor2 = 0.25 * rtol * rtol * pr[j].bb;
      q.tol2 = delta2 * s[1] > floor2 ? delta2 * s[1] : floor2;
      q.converged = 0;
      return true;
    });
    rebuild_lists(t, w, pdone);
    if (threadIdx.x == 0) {
      gs->active = active;
      gs->done = active == 0;
      gs->ticket = 0;
    }
  }
}

// d = z + beta d, h = 0 for problems still iterating; block 0 sets the while-condition
__global__ void __launch_bounds__(RED_THREADS)
bcg32_direction(ChunkTable t, const float* __restrict__ r, float* __restrict__ d, float* __restrict__ h,
                const float* __restrict__ inv_diag, const BState* ps, const int* __restrict__ pdone,
                const BGlobal* gs, cudaGraphConditionalHandle cond, int use_cond) {
  const int done = gs->done;
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, done ? 0u : 1u);
  if (done) return;
  const int nc = chunk_count(t);
  for (int ic = blockIdx.x; ic < nc; ic += gridDim.x) {
    const int c = chunk_at(t, ic);
    const int prob = t.blk_prob[c];
    if (pdone[prob]) continue;
    const float beta = (float)ps[prob].beta;
    const int64_t lo = t.blk_lo[c], hi = t.blk_hi[c];
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const float zi = inv_diag ? r[i] * inv_diag[i] : r[i];
      d[i] = fmaf(beta, d[i], zi);
      h[i] = 0.f;
    }
  }
}

// 1 on the boundary DOFs of one problem's node grid (concatenated numbering)
__global__ void mark_boundary(int64_t Nx, int64_t Ny, int64_t Nz, int64_t dof_off, unsigned char* __restrict__ mask) {
  const int64_t total = Nx * Ny * Nz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = t % Nx, y = (t / Nx) % Ny, z = t / (Nx * Ny);
    if (x == 0 || y == 0 || z == 0 || x == Nx - 1 || y == Ny - 1 || z == Nz - 1) mask[dof_off + t] = 1;
  }
}

}  // namespace fepa
