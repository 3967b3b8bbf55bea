// p-multigrid pieces (arXiv 2402.15940, Sec. 2.1): transfers between the order-p and a
// lower-order H1 space on the same mesh, applied element by element with the
// tensor-product 1D interpolation matrix (sum factorisation); diagonal (Jacobi) smoothing
// with Chebyshev acceleration; and the vector kernels of a CG preconditioned by a V-cycle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_kernels.cuh"
#include "pa_kernels.cuh"

namespace fepa {

constexpr int MG_MAXN = FEPA_MAX_ORDER + 1;

// xf = P xc: interpolate coarse nodal values to the fine nodes of every element;
// I[a][i] = coarse basis i at fine node a (nf x nc).  Shared fine nodes get the same
// value from every element that holds them (plain stores).  One element per block.
template <typename T>
__global__ void mg_prolong(int E, int nf, int nc, const int* __restrict__ gf, const int* __restrict__ gc,
                           const T* __restrict__ I, const T* __restrict__ xc, T* __restrict__ xf) {
  __shared__ T sI[MG_MAXN * MG_MAXN];
  __shared__ T s0[MG_MAXN * MG_MAXN * MG_MAXN];
  __shared__ T s1[MG_MAXN * MG_MAXN * MG_MAXN];
  const int64_t e = blockIdx.x;
  const int t = threadIdx.x, NT = blockDim.x;
  const int nc3 = nc * nc * nc, nf3 = nf * nf * nf;
  for (int k = t; k < nf * nc; k += NT) sI[k] = I[k];
  for (int k = t; k < nc3; k += NT) s0[k] = xc[gmap_dof(gc[e * nc3 + k])];
  __syncthreads();
  // x: [c][b][a'] over coarse c, b
  for (int w = t; w < nf * nc * nc; w += NT) {
    const int a = w % nf, cb = w / nf;
    T s = T(0);
    for (int i = 0; i < nc; ++i) s += sI[a * nc + i] * s0[cb * nc + i];
    s1[w] = s;
  }
  __syncthreads();
  // y: [c][b'][a']
  for (int w = t; w < nf * nf * nc; w += NT) {
    const int a = w % nf, b = (w / nf) % nf, c = w / (nf * nf);
    T s = T(0);
    for (int j = 0; j < nc; ++j) s += sI[b * nc + j] * s1[(c * nc + j) * nf + a];
    s0[w] = s;
  }
  __syncthreads();
  // z: [c'][b'][a'] -> fine DOFs
  for (int w = t; w < nf3; w += NT) {
    const int ab = w % (nf * nf), c = w / (nf * nf);
    T s = T(0);
    for (int k = 0; k < nc; ++k) s += sI[c * nc + k] * s0[k * nf * nf + ab];
    xf[gmap_dof(gf[e * nf3 + w])] = s;
  }
}

// rc += P^T rf: every fine DOF counted once (its value divided by the number of elements
// holding it), transposed interpolation, scatter-add to the coarse DOFs.  Fine essential
// entries are read as 0.
template <typename T>
__global__ void mg_restrict(int E, int nf, int nc, const int* __restrict__ gf, const int* __restrict__ gc,
                            const T* __restrict__ I, const T* __restrict__ inv_mult, const T* __restrict__ rf,
                            T* __restrict__ rc) {
  __shared__ T sI[MG_MAXN * MG_MAXN];
  __shared__ T s0[MG_MAXN * MG_MAXN * MG_MAXN];
  __shared__ T s1[MG_MAXN * MG_MAXN * MG_MAXN];
  const int64_t e = blockIdx.x;
  const int t = threadIdx.x, NT = blockDim.x;
  const int nc3 = nc * nc * nc, nf3 = nf * nf * nf;
  for (int k = t; k < nf * nc; k += NT) sI[k] = I[k];
  for (int k = t; k < nf3; k += NT) {
    const int g = gf[e * nf3 + k];
    s0[k] = g >= 0 ? rf[g] * inv_mult[g] : T(0);
  }
  __syncthreads();
  // z^T: [k][b'][a'] = sum_c' I[c'][k] s0[c'][b'][a']
  for (int w = t; w < nc * nf * nf; w += NT) {
    const int ab = w % (nf * nf), k = w / (nf * nf);
    T s = T(0);
    for (int c = 0; c < nf; ++c) s += sI[c * nc + k] * s0[c * nf * nf + ab];
    s1[w] = s;
  }
  __syncthreads();
  // y^T: [k][j][a'] = sum_b' I[b'][j] s1[k][b'][a']
  for (int w = t; w < nc * nc * nf; w += NT) {
    const int a = w % nf, j = (w / nf) % nc, k = w / (nf * nc);
    T s = T(0);
    for (int b = 0; b < nf; ++b) s += sI[b * nc + j] * s1[(k * nf + b) * nf + a];
    s0[w] = s;
  }
  __syncthreads();
  // x^T: [k][j][i] = sum_a' I[a'][i] s0[k][j][a'] -> coarse DOFs
  for (int w = t; w < nc3; w += NT) {
    const int i = w % nc, kj = w / nc;
    T s = T(0);
    for (int a = 0; a < nf; ++a) s += sI[a * nc + i] * s0[kj * nf + a];
    atomicAdd(rc + gmap_dof(gc[e * nc3 + w]), s);
  }
}

// Compiled transfers for one (fine, coarse) node count pair: several elements per block
// (NF^2 threads each), sizes known at compile time so every contraction unrolls.
template <int NF, int NC>
struct XferShape {
  static constexpr int TPE = NF * NF;
  static constexpr int NEB = (256 / TPE) > 0 ? (256 / TPE) : 1;
  static constexpr int THREADS = NEB * TPE;
};

// xf = P xc (as mg_prolong), elements blockIdx.x * NEB + threadIdx.x / NF^2
template <typename T, int NF, int NC>
__global__ void __launch_bounds__(XferShape<NF, NC>::THREADS)
mg_prolong_t(int E, const int* __restrict__ gf, const int* __restrict__ gc, const T* __restrict__ I,
             const T* __restrict__ xc, T* __restrict__ xf) {
  using S = XferShape<NF, NC>;
  constexpr int TPE = S::TPE, NEB = S::NEB, NC3 = NC * NC * NC, NF3 = NF * NF * NF;
  __shared__ T sI[NF * NC];
  __shared__ T s0[NEB][NF3];
  __shared__ T s1[NEB][NF * NC * NC];
  const int el = threadIdx.x / TPE, t = threadIdx.x - el * TPE;
  const int64_t e = (int64_t)blockIdx.x * NEB + el;
  const bool live = e < E;
  for (int k = threadIdx.x; k < NF * NC; k += S::THREADS) sI[k] = I[k];
  if (live)
    for (int k = t; k < NC3; k += TPE) s0[el][k] = xc[gmap_dof(gc[e * NC3 + k])];
  __syncthreads();
  if (live)
    for (int w = t; w < NF * NC * NC; w += TPE) {  // x: [c][b][a']
      const int a = w % NF, cb = w / NF;
      T v = T(0);
#pragma unroll
      for (int i = 0; i < NC; ++i) v += sI[a * NC + i] * s0[el][cb * NC + i];
      s1[el][w] = v;
    }
  __syncthreads();
  if (live)
    for (int w = t; w < NF * NF * NC; w += TPE) {  // y: [c][b'][a']
      const int a = w % NF, b = (w / NF) % NF, c = w / (NF * NF);
      T v = T(0);
#pragma unroll
      for (int j = 0; j < NC; ++j) v += sI[b * NC + j] * s1[el][(c * NC + j) * NF + a];
      s0[el][w] = v;
    }
  __syncthreads();
  if (live)
#pragma unroll
    for (int c = 0; c < NF; ++c) {  // z: thread (a', b') writes its column
      T v = T(0);
#pragma unroll
      for (int k = 0; k < NC; ++k) v += sI[c * NC + k] * s0[el][k * NF * NF + t];
      xf[gmap_dof(gf[e * NF3 + c * NF * NF + t])] = v;
    }
}

// rc += P^T rf (as mg_restrict)
template <typename T, int NF, int NC>
__global__ void __launch_bounds__(XferShape<NF, NC>::THREADS)
mg_restrict_t(int E, const int* __restrict__ gf, const int* __restrict__ gc, const T* __restrict__ I,
              const T* __restrict__ inv_mult, const T* __restrict__ rf, T* __restrict__ rc) {
  using S = XferShape<NF, NC>;
  constexpr int TPE = S::TPE, NEB = S::NEB, NC3 = NC * NC * NC, NF3 = NF * NF * NF;
  __shared__ T sI[NF * NC];
  __shared__ T s0[NEB][NF * NF * NC];
  __shared__ T s1[NEB][NF * NC * NC];
  const int el = threadIdx.x / TPE, t = threadIdx.x - el * TPE;
  const int64_t e = (int64_t)blockIdx.x * NEB + el;
  const bool live = e < E;
  for (int k = threadIdx.x; k < NF * NC; k += S::THREADS) sI[k] = I[k];
  __syncthreads();
  if (live) {  // z^T straight from the fine values: thread (a', b') reads its column
    T col[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      const int g = gf[e * NF3 + c * NF * NF + t];
      col[c] = g >= 0 ? rf[g] * inv_mult[g] : T(0);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      T v = T(0);
#pragma unroll
      for (int c = 0; c < NF; ++c) v += sI[c * NC + k] * col[c];
      s0[el][k * NF * NF + t] = v;
    }
  }
  __syncthreads();
  if (live)
    for (int w = t; w < NC * NC * NF; w += TPE) {  // y^T: [k][j][a']
      const int a = w % NF, j = (w / NF) % NC, k = w / (NF * NC);
      T v = T(0);
#pragma unroll
      for (int b = 0; b < NF; ++b) v += sI[b * NC + j] * s0[el][(k * NF + b) * NF + a];
      s1[el][w] = v;
    }
  __syncthreads();
  if (live)
    for (int w = t; w < NC3; w += TPE) {  // x^T: [k][j][i] -> coarse DOFs
      const int i = w % NC, kj = w / NC;
      T v = T(0);
#pragma unroll
      for (int a = 0; a < NF; ++a) v += sI[a * NC + i] * s1[el][kj * NF + a];
      atomicAdd(rc + gmap_dof(gc[e * NC3 + w]), v);
    }
}

// 1 / (number of elements holding each DOF) on a structured node grid
template <typename T>
__global__ void mg_inv_multiplicity(int nx, int ny, int nz, int p, T* __restrict__ out) {
  const int64_t Nx = (int64_t)p * nx + 1, Ny = (int64_t)p * ny + 1, Nz = (int64_t)p * nz + 1;
  const int64_t total = Nx * Ny * Nz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g[3] = {t % Nx, (t / Nx) % Ny, t / (Nx * Ny)};
    const int64_t lim[3] = {Nx - 1, Ny - 1, Nz - 1};
    int m = 1;
    for (int d = 0; d < 3; ++d)
      if (g[d] % p == 0 && g[d] > 0 && g[d] < lim[d]) m *= 2;
    out[t] = T(1) / T(m);
  }
}

// Any mesh: count[g] += 1 per element-local slot holding DOF g (count zeroed first) ...
__global__ void gmap_count(int64_t total, const int* __restrict__ gmap, int* __restrict__ count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(count + gmap_dof(gmap[t]), 1);
}

// ... then 1 / count, the inverse multiplicity used by the restriction
template <typename T>
__global__ void inv_count(int64_t N, const int* __restrict__ count, T* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = T(1) / T(count[t]);
}

// Chebyshev-accelerated Jacobi, from x = 0: start x = 0, r = b, d = D^{-1} b / theta, h = 0
template <typename T>
__global__ void cheb_start(int64_t N, const T* __restrict__ b, const T* __restrict__ invd, T inv_theta,
                           T* __restrict__ x, T* __restrict__ r, T* __restrict__ d, T* __restrict__ h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T bi = b[i];
    x[i] = T(0);
    r[i] = bi;
    d[i] = inv_theta * invd[i] * bi;
    h[i] = T(0);
  }
}

// one step after h = A d: x += d; r -= h; d = c1 d + c2 D^{-1} r; h = 0
template <typename T>
__global__ void cheb_step(int64_t N, T c1, T c2, const T* __restrict__ invd, T* __restrict__ x, T* __restrict__ r,
                          T* __restrict__ d, T* __restrict__ h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T di = d[i];
    x[i] += di;
    const T ri = r[i] - h[i];
    r[i] = ri;
    d[i] = c1 * di + c2 * invd[i] * ri;
    h[i] = T(0);
  }
}

// v[rows] = 0 (essential rows of a coarse level)
template <typename T>
__global__ void zero_rows(int64_t count, const int* __restrict__ rows, T* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    v[rows[i]] = T(0);
}

// y = a*x + y, and r = b - h (helpers of the V-cycle)
template <typename T>
__global__ void axpy(int64_t N, T a, const T* __restrict__ x, T* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

template <typename T>
__global__ void sub_to(int64_t N, const T* __restrict__ b, const T* __restrict__ h, T* __restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - h[i];
}

// out = in converted (FP64 <-> FP32 at the boundary of an FP32 V-cycle)
template <typename A, typename B>
__global__ void convert(int64_t N, const A* __restrict__ in, B* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}

// deterministic pseudo-random start vector for the eigenvalue estimate (splitmix64 of the index)
template <typename T>
__global__ void hash_fill(int64_t N, T* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (T)((double)(z >> 11) * (1.0 / 9007199254740992.0) + 0.5);
  }
}

// ---------------------------------------------------------------------------
// lambda_max(D^{-1} A) by the Lanczos process on S = D^{-1/2} A D^{-1/2} (symmetric,
// same spectrum): u_{j+1} beta_{j+1} = S u_j - alpha_j u_j - beta_j u_{j-1}.  The
// coefficients stay on the device (fixed-order block reductions, the last block writes
// them), the host takes the largest eigenvalue of the small tridiagonal matrix at the end.
// ---------------------------------------------------------------------------
constexpr int MG_LANCZOS = 10;

struct LanczosState {
  double alpha[MG_LANCZOS];
  double beta[MG_LANCZOS + 1];  // beta[0] = norm of the start vector, beta[j+1] = ||w_j||
  unsigned int ticket;
};

// beta[0] = ||v||
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
lz_norm(int64_t N, const T* __restrict__ v, LanczosState* st, double* partials) {
  // per-thread sums in T (an FP32 V-cycle's estimate needs a few digits, and FP64 products
  // would run on the slow FP64 pipe), block and grid sums in FP64
  T a0 = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    a0 += v[i] * v[i];
  double acc[1] = {(double)a0};
  double blk[1];
  block_sum<1>(acc, blk);
  if (publish_partials<1>(blk, partials, &st->ticket)) {
    double tot[1];
    final_sums<1>(partials, tot);
    if (threadIdx.x == 0) {
      st->beta[0] = sqrt(tot[0]);
      st->ticket = 0;
    }
  }
}

// u = v / beta[0]; t = D^{-1/2} u; h = 0
template <typename T>
__global__ void lz_start(int64_t N, const T* __restrict__ v, const T* __restrict__ invd, const LanczosState* st,
                         T* __restrict__ u, T* __restrict__ t, T* __restrict__ h) {
  const T sc = (T)(1.0 / st->beta[0]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T ui = sc * v[i];
    u[i] = ui;
    t[i] = sqrt(invd[i]) * ui;
    h[i] = T(0);
  }
}

// w = D^{-1/2} h - beta_j u_prev (into u_prev); alpha_j = (w, u) / (u, u);
// beta_{j+1} = ||w - alpha_j u|| = sqrt((w, w) - alpha_j (w, u)).  The measured (u, u) keeps
// rounding in u's norm from compounding (with (u, u) taken as 1 an FP32 run drifts by a
// factor ~(alpha/beta)^2 per step); a beta within rounding of zero (an invariant subspace,
// e.g. a level with a handful of free DOFs) is returned as exactly zero.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
lz_reduce(int64_t N, int j, const T* __restrict__ h, const T* __restrict__ invd, const T* __restrict__ u,
          T* __restrict__ uprev, LanczosState* st, double* partials) {
  const T bj = j > 0 ? (T)st->beta[j] : T(0);
  T a0 = T(0), a1 = T(0), a2 = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T w = sqrt(invd[i]) * h[i] - bj * uprev[i];
    const T ui = u[i];
    uprev[i] = w;
    a0 += w * ui;
    a1 += w * w;
    a2 += ui * ui;
  }
  double acc[3] = {(double)a0, (double)a1, (double)a2};
  double blk[3];
  block_sum<3>(acc, blk);
  if (publish_partials<3>(blk, partials, &st->ticket)) {
    double tot[3];
    final_sums<3>(partials, tot);
    if (threadIdx.x == 0) {
      const double a = tot[2] > 0.0 ? tot[0] / tot[2] : 0.0;
      const double b2 = tot[1] - a * tot[0];
      const double floor2 = (sizeof(T) == 4 ? 1e-5 : 1e-13) * tot[1];  // ~100x the rounding of (w, w)
      st->alpha[j] = a;
      st->beta[j + 1] = b2 > floor2 ? sqrt(b2) : 0.0;
      st->ticket = 0;
    }
  }
}

// u_next = (w - alpha_j u) / beta_{j+1} (in place of w); t = D^{-1/2} u_next; h = 0
template <typename T>
__global__ void lz_next(int64_t N, int j, const T* __restrict__ u, T* __restrict__ w, const T* __restrict__ invd,
                        const LanczosState* st, T* __restrict__ t, T* __restrict__ h) {
  const T a = (T)st->alpha[j];
  const double b = st->beta[j + 1];
  const T ib = b > 0.0 ? (T)(1.0 / b) : T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T un = (w[i] - a * u[i]) * ib;
    w[i] = un;
    t[i] = sqrt(invd[i]) * un;
    h[i] = T(0);
  }
}

// ---------------------------------------------------------------------------
// CG preconditioned by a V-cycle: scalars on the device as in cg_kernels.cuh
// ---------------------------------------------------------------------------
// r = b - h; rr = (r,r), bb = (b,b); h = 0; d = 0
__global__ void __launch_bounds__(RED_THREADS)
pcg_start(int64_t N, const double* __restrict__ b, double* __restrict__ r, double* __restrict__ h,
          double* __restrict__ d, CgState* st, double rtol2, int maxit, double* partials) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i], ri = bi - h[i];
    r[i] = ri;
    h[i] = 0.0;
    d[i] = 0.0;
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
      st->tol2 = rtol2 * tot[1];
      st->iter = 0;
      st->maxit = maxit;
      st->converged = (tot[0] <= st->tol2 && isfinite(st->tol2)) ? 1 : 0;
      st->done = st->converged || !isfinite(st->rr) || !isfinite(st->bb);  // NaN/inf: stop at once
      st->rho = 0.0;
      st->alpha = st->beta = 0.0;
      st->tick_limit = 0x7fffffff;
      st->ticket = 0;
    }
  }
}

// The iteration kernels below (and cg_dot_dh) return at once when the state says done, so an
// iteration enqueued after the stopping test (the resumable solve's last advance) changes nothing.

// rho_new = (z, r) and beta in the flexible (Polak-Ribiere) form
//   beta = (z_new, r_new - r_old) / rho_old = -alpha (z_new, h) / rho_old,  h = A d_old,
// which equals rho_new / rho_old for a fixed symmetric preconditioner and stays robust
// when the preconditioner is applied in lower precision; beta = 0 on the first step.
__global__ void __launch_bounds__(RED_THREADS)
pcg_rho(int64_t N, const double* __restrict__ z, const double* __restrict__ r, const double* __restrict__ h,
        CgState* st, double* partials) {
  if (st->done) return;
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = z[i];
    v[0] += zi * r[i];
    v[1] += zi * h[i];
  }
  double blk[2];
  block_sum<2>(v, blk);
  if (publish_partials<2>(blk, partials, &st->ticket)) {
    double tot[2];
    final_sums<2>(partials, tot);
    if (threadIdx.x == 0) {
      st->beta = st->iter == 0 ? 0.0 : -st->alpha * tot[1] / st->rho;
      st->rho = tot[0];
      st->ticket = 0;
    }
  }
}

__global__ void pcg_direction(int64_t N, const double* __restrict__ z, double* __restrict__ d, double* __restrict__ h,
                              const CgState* st) {
  if (st->done) return;
  const double beta = st->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    d[i] = beta == 0.0 ? z[i] : z[i] + beta * d[i];
    h[i] = 0.0;
  }
}

// x += alpha d; r -= alpha h; rr = (r, r); the stopping test
__global__ void __launch_bounds__(RED_THREADS)
pcg_update(int64_t N, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ d,
           const double* __restrict__ h, CgState* st, double* partials) {
  if (st->done) return;
  const double alpha = st->alpha;
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * d[i];
    const double ri = r[i] - alpha * h[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  double blk[1];
  block_sum<1>(v, blk);
  if (publish_partials<1>(blk, partials, &st->ticket)) {
    double tot[1];
    final_sums<1>(partials, tot);
    if (threadIdx.x == 0) {
      st->iter += 1;
      st->rr = tot[0];
      if (tot[0] <= st->tol2) {
        st->converged = 1;
        st->done = 1;
      } else if (st->iter >= st->maxit || !isfinite(st->rr)) {
        st->done = 1;
      }
      st->ticket = 0;
    }
  }
}

}  // namespace fepa
