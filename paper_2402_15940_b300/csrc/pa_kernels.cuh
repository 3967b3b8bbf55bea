// Partial-assembly kernels, FP64 (arXiv 2402.15940, Fig. fig_feod and Sec. 2.1-2.2).
//
//   pa_apply         y += G^T B^T D B G x, fused in one kernel per element group
//   pa_diag          diag(A) by sum factorisation (the matrix-free diagonal of Sec. 2.1)
//   qp_coords        physical quadrature points
// (geometry D and the load vector are computed in double-float: geom_df.cuh)
//
// Element -> DOF map ("gmap", the G operator) entries:
//   g >= 0                      ordinary DOF g
//   g <  0, (~g) & ESS_SKIP == 0  essential DOF ~g, this occurrence owns it
//   g <  0, (~g) & ESS_SKIP != 0  essential DOF (~g) & ESS_MASK, not the owner
// Essential DOFs are read as 0 and receive no element contribution; their owner
// occurrence adds x[g] (apply) or 1 (diagonal), which yields (I-E)A(I-E)x + Ex.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fepa {

constexpr int ESS_SKIP = 1 << 30;
constexpr int ESS_MASK = ESS_SKIP - 1;

struct CgState;  // cg_kernels.cuh

__device__ __forceinline__ int gmap_dof(int g) { return g >= 0 ? g : ((~g) & ESS_MASK); }

// ---------------------------------------------------------------------------
// D = w det J (mass) or w adj(J) adj(J)^T / det J (diffusion, 6 comps), stored
// [e][comp][q^3], point i + q*(j + q*k) (computed by geom_df.cuh); the corners of an
// element, for the quadrature-point coordinates
// ---------------------------------------------------------------------------
// vertex of corner c = i + 2j + 4k of element e: from the connectivity econn [E][8] of an
// unstructured mesh, else on the structured grid of nx x ny elements per layer (x fastest)
__device__ __forceinline__ int64_t corner_vertex(const int* __restrict__ econn, int nx, int ny, int64_t e, int c) {
  if (econn) return econn[8 * e + c];
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
  return (ex + (c & 1)) + (int64_t)(nx + 1) * ((ey + ((c >> 1) & 1)) + (int64_t)(ny + 1) * (ez + ((c >> 2) & 1)));
}

__device__ __forceinline__ void element_corners(const double* __restrict__ verts, const int* __restrict__ econn,
                                                int nx, int ny, int64_t e, double X[8][3]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t v = corner_vertex(econn, nx, ny, e, c);
    X[c][0] = verts[3 * v + 0];
    X[c][1] = verts[3 * v + 1];
    X[c][2] = verts[3 * v + 2];
  }
}

__global__ void qp_coords_kernel(int64_t E, int nx, int ny, const int* __restrict__ econn, int q,
                                 const double* __restrict__ verts, const double* __restrict__ pts,
                                 double* __restrict__ out) {
  const int64_t q3 = (int64_t)q * q * q;
  const int64_t total = E * q3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / q3;
    const int qp = (int)(t - e * q3);
    const double s = pts[qp % q], tt = pts[(qp / q) % q], u = pts[qp / (q * q)];
    double X[8][3];
    element_corners(verts, econn, nx, ny, e, X);
    double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double N = ((c & 1) ? s : 1.0 - s) * ((c & 2) ? tt : 1.0 - tt) * ((c & 4) ? u : 1.0 - u);
      x[0] += N * X[c][0];
      x[1] += N * X[c][1];
      x[2] += N * X[c][2];
    }
    out[3 * t + 0] = x[0];
    out[3 * t + 1] = x[1];
    out[3 * t + 2] = x[2];
  }
}

// ---------------------------------------------------------------------------
// structured element -> DOF map and essential flags
// ---------------------------------------------------------------------------
__global__ void build_gmap(int nx, int ny, int nz, int p, int dof_off, int* __restrict__ gmap) {
  const int n = p + 1, n3 = n * n * n;
  const int64_t Nx = (int64_t)p * nx + 1, Ny = (int64_t)p * ny + 1;
  const int64_t total = (int64_t)nx * ny * nz * n3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / n3;
    const int l = (int)(t - e * n3);
    const int a = l % n, b = (l / n) % n, c = l / (n * n);
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    gmap[t] = dof_off + (int)((p * ex + a) + Nx * ((p * ey + b) + Ny * (p * ez + c)));
  }
}

// Re-encode gmap for the essential mask (1 byte per DOF).  The owner occurrence of a
// node is the one in the element with the largest index per direction whose local
// coordinate is < p, or the last element along that direction.
__global__ void flag_gmap(int nx, int ny, int nz, int p, const unsigned char* __restrict__ ess_mask,
                          int* __restrict__ gmap) {
  const int n = p + 1, n3 = n * n * n;
  const int64_t total = (int64_t)nx * ny * nz * n3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / n3;
    const int l = (int)(t - e * n3);
    const int g = gmap_dof(gmap[t]);
    if (!ess_mask[g]) { gmap[t] = g; continue; }
    const int a = l % n, b = (l / n) % n, c = l / (n * n);
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    const bool own = (a < p || ex == nx - 1) && (b < p || ey == ny - 1) && (c < p || ez == nz - 1);
    gmap[t] = own ? ~g : ~(g | ESS_SKIP);
  }
}

// Any mesh: first[g] = the smallest element-local slot e (p+1)^3 + l holding DOF g (first
// initialised to INT_MAX); that occurrence is the owner of an essential DOF.
__global__ void gmap_first_slot(int64_t total, const int* __restrict__ gmap, int* __restrict__ first) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    atomicMin(first + gmap_dof(gmap[t]), (int)t);
}

// Any mesh: re-encode gmap for the essential mask with the owners of gmap_first_slot.
__global__ void flag_gmap_first(int64_t total, const unsigned char* __restrict__ ess_mask,
                                const int* __restrict__ first, int* __restrict__ gmap) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int g = gmap_dof(gmap[t]);
    if (!ess_mask[g]) { gmap[t] = g; continue; }
    gmap[t] = first[g] == (int)t ? ~g : ~(g | ESS_SKIP);
  }
}

__global__ void unflag_gmap(int64_t total, const int* __restrict__ gmap, int* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = gmap_dof(gmap[t]);
}

// ---------------------------------------------------------------------------
// fused operator action
// ---------------------------------------------------------------------------
template <typename T, int P, int Q, bool DIFF>
struct PaShape {
  static constexpr int N = P + 1;
  static constexpr int NC1 = DIFF ? 2 : 1;  // stage-1 arrays (B x, G x)
  static constexpr int NC2 = DIFF ? 3 : 1;  // stage-2 arrays
  static constexpr int ELEM = N * N * N + NC1 * N * N * Q + NC2 * N * Q * Q;  // values per element
  static constexpr int TPE = Q * Q;                                             // threads per element
  static constexpr int NE = (256 / TPE) > 0 ? (256 / TPE) : 1;                  // elements per block
  static constexpr int SMEM = (2 * Q * N + NE * ELEM) * (int)sizeof(T);        // bytes
};

// Each element is handled by Q*Q threads (threadIdx.x) and each block holds NE elements
// (threadIdx.y).  Stage 1 contracts the x index, stage 2 the y index, stage 3 the z index
// per (i,j) column, fused with D and the transposed z contraction in registers; the
// transposed y and x stages follow through shared memory, and the result is
// scatter-added to y (G^T).  R is the arithmetic type: double for the FP64 operator,
// float for the FP32 operator of the mixed-precision solve (D, tables, x, y all in R).
// The block's work on a tile of ne <= NE consecutive elements from e0 (called once per block by
// pa_apply, or per tile of a work list by pa_apply_tiles)
template <typename R, int P, int Q, bool DIFF>
__device__ __forceinline__ void pa_tile(int64_t e0, int ne, const int* __restrict__ gmap, const R* __restrict__ qd,
                                        const R* __restrict__ Btab, const R* __restrict__ Gtab,
                                        const R* __restrict__ x, R* __restrict__ y, const int* __restrict__ elem_prob,
                                        const int* __restrict__ prob_done) {
  using S = PaShape<R, P, Q, DIFF>;
  constexpr int n = S::N, T = S::TPE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  R* sB = smem;
  R* sG = sB + Q * n;
  R* sX = sG + Q * n + threadIdx.y * S::ELEM;
  R* S1 = sX + n * n * n;
  R* S2 = S1 + S::NC1 * n * n * Q;
  const int tid = threadIdx.x;
  const int64_t e = e0 + threadIdx.y;
  // batched operators: elements of problems that have converged do nothing
  const bool live = (int)threadIdx.y < ne && !(elem_prob && prob_done[elem_prob[e]]);
  const int* g = gmap + e * (n * n * n);

  for (int i = threadIdx.y * T + tid; i < Q * n; i += T * S::NE) {
    sB[i] = Btab[i];
    sG[i] = Gtab[i];
  }
  if (live)
    for (int l = tid; l < n * n * n; l += T) {
      const int gi = g[l];
      sX[l] = gi >= 0 ? x[gi] : R(0);
    }
  __syncthreads();

  // stage 1: S1[m][c][b][i] = sum_a {B,G}[i][a] X[c][b][a]
  if (live)
    for (int w = tid; w < n * n * Q; w += T) {
      const int i = w % Q, cb = w / Q;
      const R* xr = sX + cb * n;
      R s0 = R(0), s1 = R(0);
#pragma unroll
      for (int a = 0; a < n; ++a) {
        const R v = xr[a];
        s0 += sB[i * n + a] * v;
        if (DIFF) s1 += sG[i * n + a] * v;
      }
      S1[w] = s0;
      if (DIFF) S1[n * n * Q + w] = s1;
    }
  __syncthreads();

  // stage 2: S2[m][c][j][i] = sum_b {..}[j][b] S1[.][c][b][i]
  //   DIFF: m=0 (x:G,y:B), m=1 (x:B,y:G), m=2 (x:B,y:B); mass: m=0 (B,B)
  if (live)
    for (int w = tid; w < n * Q * Q; w += T) {
      const int i = w % Q, j = (w / Q) % Q, c = w / (Q * Q);
      const R* sb = S1 + c * n * Q + i;
      R sBB = R(0), sBG = R(0), sGB = R(0);
#pragma unroll
      for (int b = 0; b < n; ++b) {
        const R vb = sb[b * Q];
        sBB += sB[j * n + b] * vb;
        if (DIFF) {
          sBG += sG[j * n + b] * vb;
          sGB += sB[j * n + b] * sb[n * n * Q + b * Q];
        }
      }
      if (DIFF) {
        S2[w] = sGB;
        S2[n * Q * Q + w] = sBG;
        S2[2 * n * Q * Q + w] = sBB;
      } else {
        S2[w] = sBB;
      }
    }
  __syncthreads();

  // stage 3 + D + stage 3^T, one (i,j) column per thread, in registers
  if (live) {
    R c0[n], c1[n], c2[n];   // forward columns over c
    R a0[n], a1[n], a2[n];   // transposed accumulators over c
#pragma unroll
    for (int c = 0; c < n; ++c) {
      c0[c] = S2[c * Q * Q + tid];
      if (DIFF) {
        c1[c] = S2[n * Q * Q + c * Q * Q + tid];
        c2[c] = S2[2 * n * Q * Q + c * Q * Q + tid];
      }
      a0[c] = R(0);
      if (DIFF) { a1[c] = R(0); a2[c] = R(0); }
    }
    constexpr int Q3 = Q * Q * Q;
    const R* de = qd + e * (DIFF ? 6 : 1) * Q3 + tid;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      if (DIFF) {
        R u0 = R(0), u1 = R(0), u2 = R(0);
#pragma unroll
        for (int c = 0; c < n; ++c) {
          u0 += sB[k * n + c] * c0[c];  // d/dx: G_x B_y B_z
          u1 += sB[k * n + c] * c1[c];  // d/dy: B_x G_y B_z
          u2 += sG[k * n + c] * c2[c];  // d/dz: B_x B_y G_z
        }
        const R* dk = de + k * Q * Q;
        const R d00 = dk[0], d01 = dk[Q3], d02 = dk[2 * Q3], d11 = dk[3 * Q3], d12 = dk[4 * Q3],
                     d22 = dk[5 * Q3];
        const R v0 = d00 * u0 + d01 * u1 + d02 * u2;
        const R v1 = d01 * u0 + d11 * u1 + d12 * u2;
        const R v2 = d02 * u0 + d12 * u1 + d22 * u2;
#pragma unroll
        for (int c = 0; c < n; ++c) {
          a0[c] += sB[k * n + c] * v0;
          a1[c] += sB[k * n + c] * v1;
          a2[c] += sG[k * n + c] * v2;
        }
      } else {
        R u = R(0);
#pragma unroll
        for (int c = 0; c < n; ++c) u += sB[k * n + c] * c0[c];
        const R v = de[k * Q * Q] * u;
#pragma unroll
        for (int c = 0; c < n; ++c) a0[c] += sB[k * n + c] * v;
      }
    }
    // each thread overwrites only its own column of S2
#pragma unroll
    for (int c = 0; c < n; ++c) {
      S2[c * Q * Q + tid] = a0[c];
      if (DIFF) {
        S2[n * Q * Q + c * Q * Q + tid] = a1[c];
        S2[2 * n * Q * Q + c * Q * Q + tid] = a2[c];
      }
    }
  }
  __syncthreads();

  // stage 2^T: S1[0][c][b][i] = sum_j B[j][b] A0[c][j][i]
  //            S1[1][c][b][i] = sum_j G[j][b] A1[c][j][i] + B[j][b] A2[c][j][i]
  if (live)
    for (int w = tid; w < n * n * Q; w += T) {
      const int i = w % Q, b = (w / Q) % n, c = w / (n * Q);
      const R* sa = S2 + c * Q * Q + i;
      R t0 = R(0), t1 = R(0);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        t0 += sB[j * n + b] * sa[j * Q];
        if (DIFF) t1 += sG[j * n + b] * sa[n * Q * Q + j * Q] + sB[j * n + b] * sa[2 * n * Q * Q + j * Q];
      }
      S1[w] = t0;
      if (DIFF) S1[n * n * Q + w] = t1;
    }
  __syncthreads();

  // stage 1^T and scatter: y[g] += sum_i G[i][a] T0[c][b][i] + B[i][a] T1[c][b][i]
  if (live)
    for (int w = tid; w < n * n * n; w += T) {
      const int a = w % n, cb = w / n;
      const R* st = S1 + cb * Q;
      R s = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (DIFF)
          s += sG[i * n + a] * st[i] + sB[i * n + a] * st[n * n * Q + i];
        else
          s += sB[i * n + a] * st[i];
      }
      const int gi = g[w];
      if (gi >= 0) {
        atomicAdd(y + gi, s);
      } else if (!((~gi) & ESS_SKIP)) {
        atomicAdd(y + (~gi), x[~gi]);
      }
    }
}

template <typename R, int P, int Q, bool DIFF>
__global__ void __launch_bounds__(PaShape<R, P, Q, DIFF>::TPE * PaShape<R, P, Q, DIFF>::NE)
pa_apply(int E, const int* __restrict__ gmap, const R* __restrict__ qd, const R* __restrict__ Btab,
         const R* __restrict__ Gtab, const R* __restrict__ x, R* __restrict__ y, const int* __restrict__ skip,
         const int* __restrict__ elem_prob, const int* __restrict__ prob_done) {
  constexpr int NE = PaShape<R, P, Q, DIFF>::NE;
  if (skip && *skip) return;
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  pa_tile<R, P, Q, DIFF>(e0, (int)((E - e0) < NE ? (E - e0) : NE), gmap, qd, Btab, Gtab, x, y, elem_prob, prob_done);
}

// Persistent form over a work list (the batch's iteration loop), as pa_apply_f32_tiles
template <typename R, int P, int Q, bool DIFF>
__global__ void __launch_bounds__(PaShape<R, P, Q, DIFF>::TPE * PaShape<R, P, Q, DIFF>::NE)
pa_apply_tiles(const int2* __restrict__ tiles, const int* __restrict__ act, const int* __restrict__ nact,
               const int* __restrict__ gmap, const R* __restrict__ qd, const R* __restrict__ Btab,
               const R* __restrict__ Gtab, const R* __restrict__ x, R* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int count = *nact;
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const int2 tl = tiles[act[i]];
    pa_tile<R, P, Q, DIFF>(tl.x, tl.y, gmap, qd, Btab, Gtab, x, y, nullptr, nullptr);
    __syncthreads();  // (the next tile reuses the shared buffers)
  }
}

// ---------------------------------------------------------------------------
// matrix-free diagonal by sum factorisation
// diag(a,b,c) = sum_m wt_m sum_{ijk} D_m(i,j,k) X_m[i][a] Y_m[j][b] Z_m[k][c]
// with per-direction tables BB = B^2, GG = G^2, BG = B*G chosen by component m = (r,s):
// the factor in direction d is GG if r = s = d, BG if exactly one of r, s is d, else BB.
// ---------------------------------------------------------------------------
template <int P, int Q, bool DIFF>
struct DiagShape {
  static constexpr int N = P + 1;
  static constexpr int NC = DIFF ? 6 : 1;
  static constexpr int SMEM = (3 * Q * N + NC * N * Q * Q + NC * N * N * Q) * 8;
};

template <int P, int Q, bool DIFF>
__global__ void __launch_bounds__(Q * Q)
pa_diag_f64(int E, const int* __restrict__ gmap, const double* __restrict__ qd, const double* __restrict__ Btab,
            const double* __restrict__ Gtab, double* __restrict__ diag) {
  using S = DiagShape<P, Q, DIFF>;
  constexpr int n = S::N, NC = S::NC, T = Q * Q;
  extern __shared__ double smem[];
  double* tBB = smem;
  double* tGG = tBB + Q * n;
  double* tBG = tGG + Q * n;
  double* T1 = tBG + Q * n;      // [m][c][j][i]
  double* T2 = T1 + NC * n * T;  // [m][c][b][i]
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  for (int i = tid; i < Q * n; i += T) {
    tBB[i] = Btab[i] * Btab[i];
    tGG[i] = Gtab[i] * Gtab[i];
    tBG[i] = Btab[i] * Gtab[i];
  }
  __syncthreads();
  // component order xx, xy, xz, yy, yz, zz; table selector per direction: 0=BB 1=BG 2=GG
  const int selx[6] = {2, 1, 1, 0, 0, 0};
  const int sely[6] = {0, 1, 0, 2, 1, 0};
  const int selz[6] = {0, 0, 1, 0, 1, 2};
  const double wt[6] = {1.0, 2.0, 2.0, 1.0, 2.0, 1.0};
  auto tab = [&](int s) -> const double* { return s == 0 ? tBB : (s == 1 ? tBG : tGG); };

  // z: T1[m][c][j][i] = sum_k D_m(i,j,k) Z_m[k][c]
  {
    constexpr int Q3 = Q * Q * Q;
    const double* de = qd + e * NC * Q3 + tid;
    for (int m = 0; m < NC; ++m) {
      const double* Z = DIFF ? tab(selz[m]) : tBB;
      double acc[n];
#pragma unroll
      for (int c = 0; c < n; ++c) acc[c] = 0.0;
      for (int k = 0; k < Q; ++k) {
        const double dv = de[m * Q3 + k * T];
#pragma unroll
        for (int c = 0; c < n; ++c) acc[c] += dv * Z[k * n + c];
      }
#pragma unroll
      for (int c = 0; c < n; ++c) T1[(m * n + c) * T + tid] = acc[c];
    }
  }
  __syncthreads();
  // y: T2[m][c][b][i] = sum_j T1[m][c][j][i] Y_m[j][b]
  for (int w = tid; w < NC * n * n * Q; w += T) {
    const int i = w % Q, b = (w / Q) % n, mc = w / (n * Q);
    const int m = mc / n;
    const double* Y = DIFF ? tab(sely[m]) : tBB;
    const double* src = T1 + mc * T + i;
    double s = 0.0;
    for (int j = 0; j < Q; ++j) s += src[j * Q] * Y[j * n + b];
    T2[w] = s;
  }
  __syncthreads();
  // x: diag(a,b,c) = sum_m wt_m sum_i T2[m][c][b][i] X_m[i][a]
  const int* g = gmap + e * (n * n * n);
  for (int w = tid; w < n * n * n; w += T) {
    const int a = w % n, cb = w / n;
    double s = 0.0;
    for (int m = 0; m < NC; ++m) {
      const double* X = DIFF ? tab(selx[m]) : tBB;
      const double* src = T2 + (m * n * n + cb) * Q;
      double sm = 0.0;
      for (int i = 0; i < Q; ++i) sm += src[i] * X[i * n + a];
      s += (DIFF ? wt[m] : 1.0) * sm;
    }
    const int gi = g[w];
    if (gi >= 0)
      atomicAdd(diag + gi, s);
    else if (!((~gi) & ESS_SKIP))
      atomicAdd(diag + (~gi), 1.0);
  }
}

}  // namespace fepa
