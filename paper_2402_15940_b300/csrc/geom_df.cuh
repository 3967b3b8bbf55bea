// Geometry setup D (Sec. 2.2, partial assembly: the quadrature-point data stored once per
// mesh) from the trilinear map, in double-float arithmetic on the FP32 pipe.
//
// Per element the 8 corners are split once into (hi, lo) float pairs in shared memory.
// Thread (i, j) of an element forms, once, the bilinear interpolants of the element's
// bottom and top faces and their s- and t-derivatives at (s_i, t_j); along its column
// k = 0..q-1 the Jacobian is then two accurate multiply-adds per entry (the map is linear
// in u between the faces), followed by the adjugate, det J, w / det J (reciprocal by one
// Newton step) and the six symmetric components of w adj(J) adj(J)^T / det J (diffusion)
// or w det J (mass), every product an exact-FMA dot-product step.  Relative error about
// 1e-14, far inside the 1e-12 bound of the FP64 data.  The kernel writes the FP64 D and,
// when the buffers exist, its (hi, lo) copy for the double-float action and the padded
// FP32 copy for the mixed-precision operator, so no conversion pass follows.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pa_df64.cuh"
#include "pa_kernels.cuh"  // corner_vertex

namespace fepa {

// Gauss-Legendre points and weights on [0, 1] as (hi, lo) pairs, for q = 1..GQ_MAX
constexpr int GQ_MAX = FEPA_MAX_ORDER + 2;
__constant__ float c_gauss_df[(GQ_MAX + 1) * 2 * GQ_MAX * 2];

__device__ __forceinline__ dfl gauss_pt(int q, int i) {
  const int k = ((q * 2 + 0) * GQ_MAX + i) * 2;
  return {c_gauss_df[k], c_gauss_df[k + 1]};
}
__device__ __forceinline__ dfl gauss_wt(int q, int i) {
  const int k = ((q * 2 + 1) * GQ_MAX + i) * 2;
  return {c_gauss_df[k], c_gauss_df[k + 1]};
}

// Range of the double-float set-up (geometry, diagonal, load vector), checked per element by
// geom_df: element extent h >= 2^-20, coordinates |x| <= 2^20 and |x| <= 2^10 h.  Within it D is
// FP64-accurate to ~2^-38 at worst (~1e-13 on unit-cube meshes of up to 256 elements per side).
constexpr float GEOM_DF_HMIN = 1.0f / (1 << 20), GEOM_DF_RMAX = (float)(1 << 20), GEOM_DF_RATIO = 1024.f;

template <int Q>
struct GeoShape {
  static constexpr int TPE = Q * Q;
  static constexpr int NE = (256 / TPE) > 0 ? (256 / TPE) : 1;
};

// vdf: vertex coordinates as (hi, lo) pairs [nverts][3]; the corners of element e come from
// econn [E][8] when given (unstructured mesh), else from the structured vertex grid of nx x ny
// elements per layer (corner_vertex).  qd: FP64 D [E][comp][q^3]; qddf (optional): the same
// as (hi, lo) pairs; qd32 (optional): FP32 D with each component padded to d32stride values.
// bad: bit 0 set if det J <= 0 somewhere; bit 1 if an element lies outside the range where this
// double-float arithmetic keeps D to ~1e-13 (GEOM_DF_* below).  dexp (optional): atomically
// raised to the largest binary exponent of a stored D value (the double-float action's range
// check uses it).
template <int Q>
__global__ void __launch_bounds__(GeoShape<Q>::TPE * GeoShape<Q>::NE)
geom_df(int64_t E, int nx, int ny, const int* __restrict__ econn, const float2* __restrict__ vdf, int diffusion,
        double* __restrict__ qd, float2* __restrict__ qddf, float* __restrict__ qd32, int d32stride,
        int* __restrict__ bad, int* __restrict__ dexp) {
  constexpr int TPE = GeoShape<Q>::TPE, NE = GeoShape<Q>::NE, Q3 = Q * Q * Q;
  __shared__ dfl sX[NE][8][3];
  const int tid = threadIdx.x, el = threadIdx.y;
  const int64_t e = (int64_t)blockIdx.x * NE + el;
  const bool live = e < E;
  if (live) {
    for (int l = tid; l < 24; l += TPE) {  // 24 corner coordinates (q^2 may be fewer threads)
      const int c = l / 3, d = l - 3 * c;
      const int64_t v = corner_vertex(econn, nx, ny, e, c);
      const float2 xv = vdf[3 * v + d];
      sX[el][c][d] = dfl{xv.x, xv.y};
    }
  }
  __syncthreads();
  if (!live) return;
  if (tid == 0) {
    // The Jacobian comes from differences of corner coordinates held to ~2^-48 of their
    // magnitude R, so its relative error is ~2^-48 R / h for an element of extent h; det J ~ h^3
    // and adj(J) adj(J)^T ~ h^4 must also keep their low words in float range.
    float R = 0.f, h = 0.f;
    for (int c = 0; c < 8; ++c)
      for (int d = 0; d < 3; ++d) {
        R = fmaxf(R, fabsf(sX[el][c][d].h));
        h = fmaxf(h, fabsf(sX[el][c][d].h - sX[el][0][d].h));
      }
    if (!(h >= GEOM_DF_HMIN && R <= GEOM_DF_RMAX && R <= GEOM_DF_RATIO * h)) atomicOr(bad, 2);
  }
  int emax = -100000;  // largest exponent of this thread's D values
  const int i = tid % Q, j = tid / Q;
  const dfl one = {1.f, 0.f};
  const dfl s = gauss_pt(Q, i), t = gauss_pt(Q, j);
  const dfl Ns[2] = {df_sub(one, s), s}, Nt[2] = {df_sub(one, t), t};
  const dfl wij = df_mul(gauss_wt(Q, i), gauss_wt(Q, j));
  // per face z = f (corner bit 2): bilinear value F, and d/ds, d/dt, at (s, t)
  dfl F[2][3], Fs[2][3], Ft[2][3];
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dfl v = df_zero(), vs = df_zero(), vt = df_zero();
#pragma unroll
      for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
          const dfl X = sX[el][cx | (cy << 1) | (f << 2)][d];
          df_fma(v, df_mul(Ns[cx], Nt[cy]), X);
          df_fma(vs, cx ? Nt[cy] : df_neg(Nt[cy]), X);
          df_fma(vt, cy ? Ns[cx] : df_neg(Ns[cx]), X);
        }
      F[f][d] = df_norm(v);
      Fs[f][d] = df_norm(vs);
      Ft[f][d] = df_norm(vt);
    }
  // J(u) columns: d/ds = Fs0 + u (Fs1 - Fs0), d/dt likewise, d/du = F1 - F0
  dfl dS[3], dT[3], J2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dS[d] = df_sub(Fs[1][d], Fs[0][d]);
    dT[d] = df_sub(Ft[1][d], Ft[0][d]);
    J2[d] = df_sub(F[1][d], F[0][d]);
  }
  for (int k = 0; k < Q; ++k) {
    const dfl u = gauss_pt(Q, k);
    dfl J[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dfl a = Fs[0][d], b = Ft[0][d];
      df_fma(a, u, dS[d]);
      df_fma(b, u, dT[d]);
      J[d][0] = df_norm(a);
      J[d][1] = df_norm(b);
      J[d][2] = J2[d];
    }
    // adjugate: A = det(J) J^{-1}; entry = difference of two products (Dot2)
    auto m2 = [](dfl a, dfl b, dfl c, dfl d) {
      dfl r = df_zero();
      df_fma(r, a, b);
      df_fma(r, df_neg(c), d);
      return df_norm(r);
    };
    dfl A[3][3];
    A[0][0] = m2(J[1][1], J[2][2], J[1][2], J[2][1]);
    A[0][1] = m2(J[0][2], J[2][1], J[0][1], J[2][2]);
    A[0][2] = m2(J[0][1], J[1][2], J[0][2], J[1][1]);
    A[1][0] = m2(J[1][2], J[2][0], J[1][0], J[2][2]);
    A[1][1] = m2(J[0][0], J[2][2], J[0][2], J[2][0]);
    A[1][2] = m2(J[0][2], J[1][0], J[0][0], J[1][2]);
    A[2][0] = m2(J[1][0], J[2][1], J[1][1], J[2][0]);
    A[2][1] = m2(J[0][1], J[2][0], J[0][0], J[2][1]);
    A[2][2] = m2(J[0][0], J[1][1], J[0][1], J[1][0]);
    dfl det = df_zero();
    df_fma(det, J[0][0], A[0][0]);
    df_fma(det, J[0][1], A[1][0]);
    df_fma(det, J[0][2], A[2][0]);
    det = df_norm(det);
    if (!(det.h > 0.f)) atomicOr(bad, 1);
    const dfl w = df_mul(wij, gauss_wt(Q, k));
    const int qp = tid + k * TPE;
    if (!diffusion) {
      const dfl v = df_mul(w, det);
      if (v.h != 0.f) emax = max(emax, ilogbf(v.h));
      qd[e * Q3 + qp] = df_to(v);
      if (qddf) qddf[e * Q3 + qp] = make_float2(v.h, v.l);
      if (qd32) qd32[e * (int64_t)d32stride + qp] = v.h;
    } else {
      const dfl f = df_mul(w, df_recip(det));
      constexpr int ra[6] = {0, 0, 0, 1, 1, 2}, rb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        dfl g = df_zero();
#pragma unroll
        for (int c = 0; c < 3; ++c) df_fma(g, A[ra[m]][c], A[rb[m]][c]);
        const dfl v = df_mul(f, df_norm(g));
        if (v.h != 0.f) emax = max(emax, ilogbf(v.h));
        const int64_t o = (e * 6 + m) * Q3 + qp;
        qd[o] = df_to(v);
        if (qddf) qddf[o] = make_float2(v.h, v.l);
        if (qd32) qd32[(e * 6 + m) * (int64_t)d32stride + qp] = v.h;
      }
    }
  }
  if (dexp) {
    const unsigned mask = __activemask();
    const int wmax = __reduce_max_sync(mask, emax);
    if ((threadIdx.x + blockDim.x * threadIdx.y) % 32 == __ffs(mask) - 1 && wmax > *(volatile int*)dexp)
      atomicMax(dexp, wmax);
  }
}

// FP64 -> (hi, lo) pairs, any layout (vertex coordinates)
__global__ void split_pairs(int64_t count, const double* __restrict__ in, float2* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const dfl v = df_from(in[t]);
    out[t] = make_float2(v.h, v.l);
  }
}

}  // namespace fepa

namespace fepa {

// ---------------------------------------------------------------------------
// sin(pi x) in double-float.  x = k/2 + r with k = rint(2x), so |r| <= 1/4 and the
// subtraction is exact (Sterbenz); theta = pi r (pi as a (hi, lo) pair); sin theta and
// cos theta from their Taylor series about 0 by Horner's rule in t = theta^2 -- the
// coefficients of t^0..t^5 in double-float, the tail (below 1e-10 of the result for
// |theta| <= pi/4) in float; the quadrant k mod 4 picks +-sin or +-cos.  Truncation
// after t^9 (sin) and t^10 (cos): below 1e-19.
// ---------------------------------------------------------------------------
namespace dfsin {
__host__ __device__ constexpr double fact(int n) { return n <= 1 ? 1.0 : n * fact(n - 1); }
constexpr double PI = 3.14159265358979323846;
__host__ __device__ constexpr float hi(double v) { return (float)v; }
__host__ __device__ constexpr float lo(double v) { return (float)(v - (double)(float)v); }
// (hi, lo) of c at compile time
#define FEPA_DF_CONST(name, value) constexpr float name##_h = hi(value), name##_l = lo(value)
FEPA_DF_CONST(pi, PI);
FEPA_DF_CONST(s11, -1.0 / fact(11));
FEPA_DF_CONST(s9, 1.0 / fact(9));
FEPA_DF_CONST(s7, -1.0 / fact(7));
FEPA_DF_CONST(s5, 1.0 / fact(5));
FEPA_DF_CONST(s3, -1.0 / fact(3));
FEPA_DF_CONST(c10, -1.0 / fact(10));
FEPA_DF_CONST(c8, 1.0 / fact(8));
FEPA_DF_CONST(c6, -1.0 / fact(6));
FEPA_DF_CONST(c4, 1.0 / fact(4));
FEPA_DF_CONST(c2, -1.0 / fact(2));
#undef FEPA_DF_CONST
constexpr float s19 = (float)(-1.0 / fact(19)), s17 = (float)(1.0 / fact(17)), s15 = (float)(-1.0 / fact(15)),
                s13 = (float)(1.0 / fact(13));
constexpr float c20 = (float)(1.0 / fact(20)), c18 = (float)(-1.0 / fact(18)), c16 = (float)(1.0 / fact(16)),
                c14 = (float)(-1.0 / fact(14)), c12 = (float)(1.0 / fact(12));
}  // namespace dfsin

__device__ __forceinline__ dfl df_horner_head(dfl acc, dfl t, float ch, float cl) {
  return df_add(df_mul(acc, t), dfl{ch, cl});
}

__device__ __forceinline__ dfl df_sinpi(dfl x) {
  using namespace dfsin;
  const float k = rintf(2.f * x.h);
  const dfl r = df_norm(dfl{__fsub_rn(x.h, 0.5f * k), x.l});
  const dfl th = df_mul(dfl{pi_h, pi_l}, r);
  const dfl t = df_mul(th, th);
  // sin theta / theta = sum_j (-1)^j t^j / (2j+1)!
  float ts = __fmaf_rn(s19, t.h, s17);
  ts = __fmaf_rn(ts, t.h, s15);
  ts = __fmaf_rn(ts, t.h, s13);
  dfl ps = {ts, 0.f};
  ps = df_horner_head(ps, t, s11_h, s11_l);
  ps = df_horner_head(ps, t, s9_h, s9_l);
  ps = df_horner_head(ps, t, s7_h, s7_l);
  ps = df_horner_head(ps, t, s5_h, s5_l);
  ps = df_horner_head(ps, t, s3_h, s3_l);
  ps = df_horner_head(ps, t, 1.f, 0.f);
  const dfl sn = df_mul(th, ps);
  // cos theta = sum_j (-1)^j t^j / (2j)!
  float tc = __fmaf_rn(c20, t.h, c18);
  tc = __fmaf_rn(tc, t.h, c16);
  tc = __fmaf_rn(tc, t.h, c14);
  tc = __fmaf_rn(tc, t.h, c12);
  dfl pc = {tc, 0.f};
  pc = df_horner_head(pc, t, c10_h, c10_l);
  pc = df_horner_head(pc, t, c8_h, c8_l);
  pc = df_horner_head(pc, t, c6_h, c6_l);
  pc = df_horner_head(pc, t, c4_h, c4_l);
  pc = df_horner_head(pc, t, c2_h, c2_l);
  pc = df_horner_head(pc, t, 1.f, 0.f);
  const int quad = ((int)k) & 3;
  const dfl v = (quad & 1) ? pc : sn;
  return (quad & 2) ? df_neg(v) : v;
}

// ---------------------------------------------------------------------------
// load vector b[g] += sum over points of w det J f phi_g (transposed stages), in
// double-float: f given per point (f_qp, FP64) or scale sin(pi x) sin(pi y) sin(pi z).
// Several elements per block; thread (i, j) walks its column k as in geom_df.
// ---------------------------------------------------------------------------
template <int P, int Q>
struct RhsDfShape {
  static constexpr int N = P + 1, TPE = Q * Q;
  static constexpr int NE = (256 / TPE) > 0 ? (256 / TPE) : 1;
  static constexpr int PER = N * TPE + N * N * Q;  // S2 [c][j][i] + S1 [c][b][i]
  static constexpr int SMEM = NE * (PER + 24) * 8;
};

template <int P, int Q>
__global__ void __launch_bounds__(RhsDfShape<P, Q>::TPE * RhsDfShape<P, Q>::NE)
pa_rhs_df(int64_t E, int nx, int ny, const int* __restrict__ econn, const float2* __restrict__ vdf,
          const int* __restrict__ gmap, const double* __restrict__ f_qp, double scale, double bscale,
          double* __restrict__ b) {
  using S = RhsDfShape<P, Q>;
  using T = TabDf<P, Q>;
  constexpr int n = S::N, TPE = S::TPE, NE = S::NE;
  extern __shared__ __align__(16) unsigned char smem_rh[];
  dfl* base = reinterpret_cast<dfl*>(smem_rh);
  const int tid = threadIdx.x, el = threadIdx.y;
  dfl* sX = base + el * (S::PER + 24);  // corners [8][3]
  dfl* S2 = sX + 24;
  dfl* S1 = S2 + n * TPE;
  const int64_t e = (int64_t)blockIdx.x * NE + el;
  const bool live = e < E;
  if (live) {
    for (int l = tid; l < 24; l += TPE) {
      const int c = l / 3, d = l - 3 * c;
      const int64_t v = corner_vertex(econn, nx, ny, e, c);
      const float2 xv = vdf[3 * v + d];
      sX[l] = dfl{xv.x, xv.y};
    }
  }
  __syncthreads();
  if (live && tid < TPE) {
    const int i = tid % Q, j = tid / Q;
    const dfl one = {1.f, 0.f};
    const dfl s = gauss_pt(Q, i), t = gauss_pt(Q, j);
    const dfl Ns[2] = {df_sub(one, s), s}, Nt[2] = {df_sub(one, t), t};
    const dfl wij = df_mul(gauss_wt(Q, i), gauss_wt(Q, j));
    dfl F[2][3], Fs[2][3], Ft[2][3];
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        dfl v = df_zero(), vs = df_zero(), vt = df_zero();
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
          for (int cx = 0; cx < 2; ++cx) {
            const dfl X = sX[3 * (cx | (cy << 1) | (f << 2)) + d];
            df_fma(v, df_mul(Ns[cx], Nt[cy]), X);
            df_fma(vs, cx ? Nt[cy] : df_neg(Nt[cy]), X);
            df_fma(vt, cy ? Ns[cx] : df_neg(Ns[cx]), X);
          }
        F[f][d] = df_norm(v);
        Fs[f][d] = df_norm(vs);
        Ft[f][d] = df_norm(vt);
      }
    dfl dF[3], dS[3], dT[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dF[d] = df_sub(F[1][d], F[0][d]);
      dS[d] = df_sub(Fs[1][d], Fs[0][d]);
      dT[d] = df_sub(Ft[1][d], Ft[0][d]);
    }
    dfl acc[n];
#pragma unroll
    for (int c = 0; c < n; ++c) acc[c] = df_zero();
    for (int k = 0; k < Q; ++k) {
      const dfl u = gauss_pt(Q, k);
      dfl J[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        dfl a = Fs[0][d], bb = Ft[0][d];
        df_fma(a, u, dS[d]);
        df_fma(bb, u, dT[d]);
        J[d][0] = df_norm(a);
        J[d][1] = df_norm(bb);
        J[d][2] = dF[d];
      }
      dfl det = df_zero();  // expansion along the first column: sum_d J[d][0] cofactor
      {
        dfl c0 = df_zero(), c1 = df_zero(), c2 = df_zero();
        df_fma(c0, J[1][1], J[2][2]);
        df_fma(c0, df_neg(J[1][2]), J[2][1]);
        df_fma(c1, J[0][2], J[2][1]);
        df_fma(c1, df_neg(J[0][1]), J[2][2]);
        df_fma(c2, J[0][1], J[1][2]);
        df_fma(c2, df_neg(J[0][2]), J[1][1]);
        df_fma(det, J[0][0], df_norm(c0));
        df_fma(det, J[1][0], df_norm(c1));
        df_fma(det, J[2][0], df_norm(c2));
      }
      dfl f;
      if (f_qp) {
        f = df_from(f_qp[e * (Q * Q * Q) + tid + k * TPE]);
      } else {
        dfl xp[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          dfl v = F[0][d];
          df_fma(v, u, dF[d]);
          xp[d] = df_norm(v);
        }
        f = df_mul(df_mul(df_from(scale), df_sinpi(xp[0])), df_mul(df_sinpi(xp[1]), df_sinpi(xp[2])));
      }
      const dfl v = df_mul(df_mul(df_mul(wij, gauss_wt(Q, k)), df_norm(det)), f);
#pragma unroll
      for (int c = 0; c < n; ++c) df_fma(acc[c], T::B(k, c), v);
    }
#pragma unroll
    for (int c = 0; c < n; ++c) S2[c * TPE + tid] = df_norm(acc[c]);
  }
  __syncthreads();
  if (live)  // y^T: S1[c][b][i] = sum_j B[j][b] S2[c][j][i]
    for (int w = tid; w < n * n * Q; w += TPE) {
      const int i = w % Q, bb = (w / Q) % n, c = w / (n * Q);
      dfl s = df_zero();
#pragma unroll
      for (int j = 0; j < Q; ++j) df_fma(s, T::B(j, bb), S2[c * TPE + j * Q + i]);
      S1[w] = df_norm(s);
    }
  __syncthreads();
  if (live) {  // x^T and scatter
    const int* g = gmap + e * (n * n * n);
    for (int w = tid; w < n * n * n; w += TPE) {
      const int a = w % n, cb = w / n;
      dfl s = df_zero();
#pragma unroll
      for (int i = 0; i < Q; ++i) df_fma(s, T::B(i, a), S1[cb * Q + i]);
      atomicAdd(b + gmap_dof(g[w]), df_to(s) * bscale);
    }
  }
}

}  // namespace fepa
