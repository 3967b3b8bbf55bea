// FP64-accurate partial-assembly action evaluated on the FP32 pipe (the operator
// y = G^T B^T D B G x of Fig. fig_feod, arXiv 2402.15940).
//
// On this GPU the FP64 pipe issues 2 DFMA per cycle per SM against 128 FFMA, so the FP64
// operator is bound by the FP64 pipe (the native kernel keeps it ~93 % busy).  Here every
// value is an unevaluated sum of two floats (hi + lo, about 48 significant bits) and every
// multiply-add of the contractions is an accurate dot-product step: the product of the
// high parts is split exactly by an FMA, the cross terms are added by FMAs, and the
// running sum is kept exact by TwoSum with the rounding errors collected in the low word
// (the "Dot2" scheme of Ogita, Rump and Oishi).  That is ~12 FP32 instructions per FP64-
// accurate multiply-add, several times the DFMA throughput, with a relative error of
// about 2^-48 per contraction -- far inside the 1e-12 parity bound of the FP64 action.
// x and y stay FP64 in memory: x is split into (hi, lo) as it is gathered and the element
// result is recombined in FP64 and scattered with FP64 atomics.  D is read as (hi, lo)
// float pairs (8 bytes per value, as FP64) split once from the FP64 D by split_to_df:
// converting D in the hot loop would put ~4 FP64-pipe instructions per stored value on
// the very pipe this kernel exists to avoid.
// Stage order and thread mapping follow the FP32 kernel (pa_tma_f32.cuh, variant 1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pa_tma_f32.cuh"

namespace fepa {

struct __align__(8) dfl {
  float h, l;
};

// binary exponents for the double-float action's range test (pa_apply_df): a product of
// exponent e has error terms near 2^(e-48) that must stay normal floats (e >= -70 keeps 8
// exponents to spare), sums must not overflow (e <= 100), and the gathered values' own low
// words must stay normal (exponent >= -90)
constexpr int DF_EXP_LO = -70, DF_EXP_HI = 100, DF_XEXP_LO = -90;

// biased binary exponent field of a double (0 for zero and subnormals, 2047 for inf/NaN)
__device__ __forceinline__ int f64_exp_field(double v) {
  return (int)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff;
}

__device__ __forceinline__ dfl df_from(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ dfl df_zero() { return {0.f, 0.f}; }
__device__ __forceinline__ dfl df_ld(const float2* p) {
  const float2 v = __ldg(p);
  return {v.x, v.y};
}

// acc += t * x, accurately (TwoProd by FMA for the high parts, cross terms by FMA,
// TwoSum for the running sum, errors into the low word)
__device__ __forceinline__ void df_fma(dfl& acc, dfl t, dfl x) {
  const float p = __fmul_rn(t.h, x.h);
  float e = __fmaf_rn(t.h, x.h, -p);
  e = __fmaf_rn(t.h, x.l, e);
  e = __fmaf_rn(t.l, x.h, e);
  const float s = __fadd_rn(acc.h, p);
  const float bv = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

// a * b (Dekker's product with the exact FMA split of the high words; cross terms by FMA)
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float s = __fadd_rn(p, e);
  return {s, __fsub_rn(e, __fsub_rn(s, p))};
}

// a + b (TwoSum of the high words, low words added, renormalised: Dekker's addition;
// absolute error ~2^-48 (|a| + |b|))
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bv = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bv)), __fsub_rn(b.h, bv));
  const float t = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float r = __fadd_rn(s, t);
  return {r, __fsub_rn(t, __fsub_rn(r, s))};
}
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// renormalise so that |lo| <= ulp(hi)/2 (Fast2Sum; valid as |lo| is far below |hi|)
__device__ __forceinline__ dfl df_norm(dfl a) {
  const float s = __fadd_rn(a.h, a.l);
  return {s, __fsub_rn(a.l, __fsub_rn(s, a.h))};
}

// 1 / b: the correctly rounded float reciprocal of the high word refined by one Newton
// step carried in double-float (r = r0 + r0 (1 - b r0)); relative error ~2^-46
__device__ __forceinline__ dfl df_recip(dfl b) {
  const float r0 = __frcp_rn(b.h);
  dfl e = {1.f, 0.f};
  df_fma(e, df_neg(b), dfl{r0, 0.f});  // 1 - b r0, accurately
  return df_norm(dfl{r0, __fmul_rn(r0, df_norm(e).h)});
}

// ---------------------------------------------------------------------------
// two double-float values in packed form: (h.x, l.x) and (h.y, l.y).  Each operation below
// is the scalar one of the same name applied to both halves with packed FP32 instructions
// (__fadd2_rn, __fmul2_rn, __ffma2_rn: per component the rounding of the scalar
// instruction), so the results are bit-identical to two scalar calls in half the
// instructions.
// ---------------------------------------------------------------------------
struct __align__(16) df2 {
  float2 h, l;
};

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, f2neg(b)); }
__device__ __forceinline__ df2 df2_zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ df2 df2_pack(dfl a, dfl b) { return {make_float2(a.h, b.h), make_float2(a.l, b.l)}; }
__device__ __forceinline__ dfl df2_x(df2 a) { return {a.h.x, a.l.x}; }
__device__ __forceinline__ dfl df2_y(df2 a) { return {a.h.y, a.l.y}; }

// acc += t * x (df_fma on both halves)
__device__ __forceinline__ void df2_fma(df2& acc, float2 th, float2 tl, float2 xh, float2 xl) {
  const float2 p = __fmul2_rn(th, xh);
  float2 e = __ffma2_rn(th, xh, f2neg(p));
  e = __ffma2_rn(th, xl, e);
  e = __ffma2_rn(tl, xh, e);
  const float2 s = __fadd2_rn(acc.h, p);
  const float2 bv = f2sub(s, acc.h);
  const float2 err = __fadd2_rn(f2sub(acc.h, f2sub(s, bv)), f2sub(p, bv));
  acc.h = s;
  acc.l = __fadd2_rn(acc.l, __fadd2_rn(err, e));
}

// a + b (df_add on both halves)
__device__ __forceinline__ df2 df2_add(df2 a, df2 b) {
  const float2 s = __fadd2_rn(a.h, b.h);
  const float2 bv = f2sub(s, a.h);
  const float2 e = __fadd2_rn(f2sub(a.h, f2sub(s, bv)), f2sub(b.h, bv));
  const float2 t = __fadd2_rn(e, __fadd2_rn(a.l, b.l));
  const float2 r = __fadd2_rn(s, t);
  return {r, f2sub(t, f2sub(r, s))};
}

// renormalise (df_norm on both halves)
__device__ __forceinline__ df2 df2_norm(df2 a) {
  const float2 s = __fadd2_rn(a.h, a.l);
  return {s, f2sub(a.l, f2sub(s, a.h))};
}

// (a + b, a - b) of two scalars' double-float values in one packed addition
__device__ __forceinline__ df2 df2_sumdiff(dfl a, dfl b) {
  return df2_add(df2_pack(a, a), df2{make_float2(b.h, -b.h), make_float2(b.l, -b.l)});
}

// FP64 1D tables of every compiled (P, Q) as double-float values in the pair layout of the FP32
// tables (tab32_offset, pa_tma_f32.cuh), each pair as a hi pair then a lo pair: rows
// R[kp][a] = (T(2kp, a), T(2kp+1, a)) and columns C[k][ap] = (T(k, 2ap), T(k, 2ap+1)) for
// T = B, G, so that the packed direct contractions take a table pair as one operand
__constant__ float2 c_tabdf[2 * TAB32_PAIRS];

// Even/odd form of the 1D contractions (q = p + 2).  The GLL nodes and the Gauss points are
// symmetric about 1/2, so B(Q-1-q, n-1-a) = B(q, a) and G(Q-1-q, n-1-a) = -G(q, a).  For a
// matrix M with M(NO-1-o, NI-1-i) = S M(o, i) (S = +1 for B and B^T, -1 for G and G^T):
// with x+_i = x_i + x_{NI-1-i}, x-_i = x_i - x_{NI-1-i} (i < NI/2) and x_mid the middle
// input when NI is odd,
//   E_o = sum_i e(o,i) x+_i + M(o, mid) x_mid,  e(o,i) = (M(o,i) + M(o,NI-1-i)) / 2
//   O_o = sum_i d(o,i) x-_i,                      d(o,i) = (M(o,i) - M(o,NI-1-i)) / 2
//   y_o = E_o + O_o,  y_{NO-1-o} = S (E_o - O_o)   (o < NO/2),
// and for odd NO the middle output is sum_i M(mid, i) x(+ or -)_i (+ M(mid, mid) x_mid
// when S = +1): half the multiply-adds of the direct form for n + Q extra additions.
// E_o and O_o are accumulated side by side as one packed pair (df2 below), so their tables are
// stored as pairs too.  Tables per q = p + 2 slot (p - 1): matrices 0 B, 1 G (Q x n), 2 B^T,
// 3 G^T (n x Q), each EO_MAT entries of a hi pair and a lo pair (float2 each):
// (e(o,i), d(o,i)) for o < NO/2, i < NI/2, then (M(o, mid), 0) for o < NO/2, then
// (M(mid, i), 0) for i <= NI/2.
constexpr int EO_MAT = 30;
__constant__ float2 c_tabeo[FEPA_MAX_ORDER * 4 * EO_MAT * 2];

template <int P, int MAT>
struct TabEo {
  static constexpr int NO = MAT < 2 ? P + 2 : P + 1, NI = MAT < 2 ? P + 1 : P + 2;
  static constexpr int HO = NO / 2, HI = NI / 2;
  static_assert(HO * HI + HO + HI + 1 <= EO_MAT, "even/odd table size");
  static constexpr int OFF = ((P - 1) * 4 + MAT) * EO_MAT * 2;
  static __device__ __forceinline__ float2 hp(int k) { return c_tabeo[OFF + 2 * k]; }
  static __device__ __forceinline__ float2 lp(int k) { return c_tabeo[OFF + 2 * k + 1]; }
  // (e(o,i), d(o,i)) as hi and lo pairs
  static __device__ __forceinline__ float2 EDh(int o, int i) { return hp(o * HI + i); }
  static __device__ __forceinline__ float2 EDl(int o, int i) { return lp(o * HI + i); }
  static __device__ __forceinline__ dfl E(int o, int i) { return {EDh(o, i).x, EDl(o, i).x}; }
  static __device__ __forceinline__ dfl D(int o, int i) { return {EDh(o, i).y, EDl(o, i).y}; }
  static __device__ __forceinline__ dfl MC(int o) { return {hp(HO * HI + o).x, lp(HO * HI + o).x}; }
  static __device__ __forceinline__ dfl MR(int i) { return {hp(HO * HI + HO + i).x, lp(HO * HI + HO + i).x}; }
};

// the mirrored input pairs packed as (x+_i, x-_i)
template <int NI>
__device__ __forceinline__ void eo_split2(const dfl (&x)[NI], df2 (&xpm)[NI / 2]) {
#pragma unroll
  for (int i = 0; i < NI / 2; ++i) xpm[i] = df2_sumdiff(x[i], x[NI - 1 - i]);
}

// y = M x from the packed split input: E_o and O_o accumulate as one pair; the mirrored
// outputs E_o + O_o and E_o - O_o come from one packed addition
template <class TE, int S>
__device__ __forceinline__ void eo_apply2(const df2 (&xpm)[TE::HI], dfl xmid, dfl (&y)[TE::NO]) {
  constexpr int HO = TE::HO, HI = TE::HI, NO = TE::NO, NI = TE::NI;
#pragma unroll
  for (int o = 0; o < HO; ++o) {
    df2 ed = df2_zero();
#pragma unroll
    for (int i = 0; i < HI; ++i) df2_fma(ed, TE::EDh(o, i), TE::EDl(o, i), xpm[i].h, xpm[i].l);
    dfl e = df2_x(ed);
    if (NI % 2) df_fma(e, TE::MC(o), xmid);
    const df2 r = df2_sumdiff(e, df2_y(ed));  // (e + d, e - d)
    y[o] = df2_x(r);
    y[NO - 1 - o] = S > 0 ? df2_y(r) : df_neg(df2_y(r));
  }
  if (NO % 2) {
    dfl m = df_zero();
#pragma unroll
    for (int i = 0; i < HI; ++i) df_fma(m, TE::MR(i), S > 0 ? df2_x(xpm[i]) : df2_y(xpm[i]));
    if (S > 0 && NI % 2) df_fma(m, TE::MR(HI), xmid);
    y[HO] = df_norm(m);
  }
}

// v = D u at two quadrature points ka (.x) and kb (.y) of a stage-3 column, packed: D at dE as
// (hi, lo) pairs, point stride PS, component stride DS; diffusion the symmetric 3 x 3 D of each
// point times (u0, u1, u2), mass D u0 (per component the scalar steps of the single-point form)
template <bool DIFF, int NC, int PS, int DS>
__device__ __forceinline__ void df2_dpoint(const float2* __restrict__ dE, int ka, int kb, df2 u0, df2 u1, df2 u2,
                                           df2& v0, df2& v1, df2& v2) {
  float2 dh[NC], dl[NC];
#pragma unroll
  for (int m = 0; m < NC; ++m) {
    const float2 da = __ldg(dE + ka * PS + m * DS), db = __ldg(dE + kb * PS + m * DS);
    dh[m] = make_float2(da.x, db.x);
    dl[m] = make_float2(da.y, db.y);
  }
  v0 = df2_zero();
  if (DIFF) {
    const int i1 = 1 % NC, i2 = 2 % NC, i3 = 3 % NC, i4 = 4 % NC, i5 = 5 % NC;
    v1 = df2_zero();
    v2 = df2_zero();
    df2_fma(v0, dh[0], dl[0], u0.h, u0.l);
    df2_fma(v0, dh[i1], dl[i1], u1.h, u1.l);
    df2_fma(v0, dh[i2], dl[i2], u2.h, u2.l);
    df2_fma(v1, dh[i1], dl[i1], u0.h, u0.l);
    df2_fma(v1, dh[i3], dl[i3], u1.h, u1.l);
    df2_fma(v1, dh[i4], dl[i4], u2.h, u2.l);
    df2_fma(v2, dh[i2], dl[i2], u0.h, u0.l);
    df2_fma(v2, dh[i4], dl[i4], u1.h, u1.l);
    df2_fma(v2, dh[i5], dl[i5], u2.h, u2.l);
    v1 = df2_norm(v1);
    v2 = df2_norm(v2);
  } else {
    df2_fma(v0, dh[0], dl[0], u0.h, u0.l);
  }
  v0 = df2_norm(v0);
}

template <int P, int Q>
struct TabDf {
  static constexpr int N = P + 1, QH = (Q + 1) / 2, NH = (N + 1) / 2;
  static constexpr int BR = 2 * tab32_offset(P, Q), GR = BR + 2 * QH * N, BC = GR + 2 * QH * N, GC = BC + 2 * Q * NH;
  // packed: hi and lo pairs of rows (2kp, 2kp+1) at column a, of columns (2ap, 2ap+1) at row k
  static __device__ __forceinline__ float2 Brh(int kp, int a) { return c_tabdf[BR + 2 * (kp * N + a)]; }
  static __device__ __forceinline__ float2 Brl(int kp, int a) { return c_tabdf[BR + 2 * (kp * N + a) + 1]; }
  static __device__ __forceinline__ float2 Grh(int kp, int a) { return c_tabdf[GR + 2 * (kp * N + a)]; }
  static __device__ __forceinline__ float2 Grl(int kp, int a) { return c_tabdf[GR + 2 * (kp * N + a) + 1]; }
  static __device__ __forceinline__ float2 Bch(int k, int ap) { return c_tabdf[BC + 2 * (k * NH + ap)]; }
  static __device__ __forceinline__ float2 Bcl(int k, int ap) { return c_tabdf[BC + 2 * (k * NH + ap) + 1]; }
  static __device__ __forceinline__ float2 Gch(int k, int ap) { return c_tabdf[GC + 2 * (k * NH + ap)]; }
  static __device__ __forceinline__ float2 Gcl(int k, int ap) { return c_tabdf[GC + 2 * (k * NH + ap) + 1]; }
  // scalar entries
  static __device__ __forceinline__ dfl B(int i, int a) {
    return (i & 1) ? dfl{Brh(i >> 1, a).y, Brl(i >> 1, a).y} : dfl{Brh(i >> 1, a).x, Brl(i >> 1, a).x};
  }
  static __device__ __forceinline__ dfl G(int i, int a) {
    return (i & 1) ? dfl{Grh(i >> 1, a).y, Grl(i >> 1, a).y} : dfl{Grh(i >> 1, a).x, Grl(i >> 1, a).x};
  }
};

// one element group per block (as many elements as fill ~256 threads), D read directly
// Launch shape of the double-float action: NE_DIV 1 the block of the FP32 layout's NE0
// elements, 2 half as many (FP64 variant 2: more, smaller blocks, for small meshes and the
// batch's groups; chosen by timing per (p, q, form, size class) and per batch group)
template <int P, int Q, bool DIFF, int NE_DIV = 1>
struct DfShape {
  using L = F32Layout<P, Q, DIFF>;
  static constexpr int N = P + 1, TPE = Q * Q;
  static constexpr int NE = (L::NE0 / NE_DIV) > 0 ? (L::NE0 / NE_DIV) : 1;
  static constexpr int SMEM = NE * (L::XSZ + L::WORK) * 8;
};

// PF: L2 prefetch of the group's D and map at block start (as in pa_tma_f32.cuh; 4-9 %).
// MINB: resident blocks per SM the register allocation must allow (0: no constraint);
// KU: unroll of the stage-3 quadrature loop (Q = fully unrolled).  Measured on B300 with
// the scalar arithmetic: for diffusion from p = 4 on, a fully unrolled stage 3 held 100-255
// registers and one or two blocks per SM; with the loop rolled (tables read per k from
// constant memory) and two blocks per SM guaranteed, p = 4 ran 1.08x, p = 6 2.7x and p = 8
// 2.2x faster.  Lower orders and the mass form are fastest with no constraint (an explicit
// minimum of 1 lets the allocator take up to 255 registers: 1.1-2x slower).  With the
// packed pairs (two blocks per SM kept), a fully unrolled stage 3 is faster again for
// diffusion p = 4, 5, 6 (4 %, 9 %, 2 %) and mass p = 6, 8 (15 %, 13 %); p = 7 equal, p = 8
// 16 % slower (rolled there).
// EO3: stage 3 (z, D, z^T) also in even/odd form over mirrored point pairs (q = p + 2), in
// packed pairs.  Measured (stand-alone launches against the scalar build): diffusion p = 4
// 12 %, p = 5 9 %, p = 6 19 %, p = 7 24 %, p = 8 32 % faster; at p = 2 13 % slower than the
// direct stage 3 (kept there).  (Before the packed form it was slower at p = 5, 6, 7.)
template <int P, int Q, bool DIFF>
struct DfTune {
  static constexpr int MINB = (DIFF && P >= 4) ? 2 : 0;
  static constexpr int KU = (DIFF && P >= 7) ? 1 : Q;
  static constexpr bool EO3 = DIFF ? (P >= 3) : (P >= 2);
  // PK3: the direct stage 3 (where EO3 is not used) in packed pairs over point pairs.
  // Measured: diffusion q = p + 2, p = 2 6 % and p = 1 1 % faster; mass p = 1 5 % and
  // q = p + 1 3 % slower (more registers: 76-84 instead of 48-64), scalar there.
  static constexpr bool PK3 = DIFF && Q == P + 2 && P <= 2;
};

// The block's work on one tile of ne <= NE consecutive elements starting at e0 (called once per
// block by pa_apply_df, or per tile of a work list by pa_apply_df_tiles)
template <int P, int Q, bool DIFF, int KU = DfTune<P, Q, DIFF>::KU, int PF = 2, int NE_DIV = 1>
__device__ __forceinline__ void df_tile(int64_t e0, int ne, const int* __restrict__ gmap,
                                        const float2* __restrict__ qd, const double* __restrict__ x,
                                        double* __restrict__ y, const int* __restrict__ elem_prob,
                                        const int* __restrict__ prob_done, int dexp) {
  using S = DfShape<P, Q, DIFF, NE_DIV>;
  using L = typename S::L;
  using T = TabDf<P, Q>;
  constexpr int n = S::N, TPE = S::TPE, NE = S::NE;
  constexpr int DQ1 = Q | 1;  // S1 line stride (odd), within the FP32 layout's S1 component size
  // even/odd line contractions (tables for q = p + 2; at p = 1 the extra additions cost more
  // than the halved multiply-adds save: measured 2 % slower there, 2-35 % faster from p = 2)
  constexpr bool EO = (Q == P + 2) && P >= 2;
  using EB = TabEo<P, 0>;
  using EG = TabEo<P, 1>;
  using EBT = TabEo<P, 2>;
  using EGT = TabEo<P, 3>;
  static_assert(DQ1 * n * n <= L::S1C, "S1 component size");
  extern __shared__ __align__(16) unsigned char smem_df[];
  dfl* sXall = reinterpret_cast<dfl*>(smem_df);
  dfl* sWall = sXall + NE * L::XSZ;
  const int tid = threadIdx.x, el = threadIdx.y;
  // L2 prefetch of the group's D and map (batched problems: not when the problems of the
  // group's first and last elements have converged)
  if (PF > 0 && tid == 0 && el == 0 &&
      !(elem_prob && prob_done[elem_prob[e0]] && prob_done[elem_prob[e0 + ne - 1]]))
    prefetch_group<PF>(qd + e0 * (L::NC * L::Q3), (size_t)ne * L::NC * L::Q3 * 8u, gmap + e0 * (n * n * n),
                       ne * n * n * n);
  // batched problems: the elements of a converged problem do no work
  const bool live = el < ne && !(elem_prob && prob_done[elem_prob[e0 + el]]);
  dfl* sX = sXall + el * L::XSZ;
  dfl* S1 = sWall + el * L::WORK;
  dfl* S2 = S1 + L::NC1 * L::S1C;
  const int* g = gmap + (e0 + el) * (n * n * n);
  constexpr int GR = (n * n * n + TPE - 1) / TPE;
  // Exponent range: a double-float value keeps ~48 bits only while its low word and the
  // error terms of its products stay normal floats.  The block's largest |x| (exponent bx)
  // is found with the gather; if bx, or the products' scale bx + dexp (dexp: D's largest
  // exponent), leaves the DF_EXP_* range, x is re-gathered times 2^-(bx + dexp) and the element
  // results are multiplied back by 2^(bx + dexp) in FP64 -- exact powers of two.
  constexpr int NW = (TPE * NE + 31) / 32;
  __shared__ int s_wexp[NW];
  int bx_thread = 0;  // largest biased exponent field of this thread's x values (0: none)
  if (live) {
    // gather: all map loads first, then all x loads, so the dependent pairs overlap
    int gi[GR];
    double xv[GR];
#pragma unroll
    for (int r = 0; r < GR; ++r) {
      const int l = tid + r * TPE;
      gi[r] = l < n * n * n ? __ldg(g + l) : -1;
    }
#pragma unroll
    for (int r = 0; r < GR; ++r) xv[r] = gi[r] >= 0 ? __ldg(x + gi[r]) : 0.0;
#pragma unroll
    for (int r = 0; r < GR; ++r) {
      const int l = tid + r * TPE;
      if (l < n * n * n) sX[(l / n) * L::XL + l % n] = df_from(xv[r]);
      bx_thread = max(bx_thread, f64_exp_field(xv[r]));
    }
  }
  {
    const int lin = tid + TPE * el, wbase = lin & ~31;  // (the last warp may be partial)
    const unsigned wmask = (TPE * NE - wbase >= 32) ? 0xffffffffu : ((1u << (TPE * NE - wbase)) - 1u);
    const int wx = __reduce_max_sync(wmask, bx_thread);
    if ((lin & 31) == 0) s_wexp[lin >> 5] = wx;
  }
  __syncthreads();
  double yscale = 1.0;     // element results times this ...
  bool rescaled = false;   // ... when the block rescaled x (block-uniform)
  {
    int bf = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) bf = max(bf, s_wexp[w]);
    const int bx = bf - 1023, sh = bx + dexp;
    if (bf != 0 && (sh > DF_EXP_HI || sh < DF_EXP_LO || bx > DF_EXP_HI || bx < DF_XEXP_LO)) {
      rescaled = true;
      // rare: rescale (uniform over the block, so the barrier below is reached by all)
      yscale = ldexp(1.0, sh);
      if (live) {
#pragma unroll
        for (int r = 0; r < GR; ++r) {
          const int l = tid + r * TPE;
          if (l < n * n * n) {
            const int gg = __ldg(g + l);  // (essential DOFs enter as 0, as in the gather above)
            sX[(l / n) * L::XL + l % n] = df_from(gg >= 0 ? ldexp(__ldg(x + gg), -sh) : 0.0);
          }
        }
      }
      __syncthreads();
    }
  }

  // stage 1 (x): line (b,c) -> S1[m][c][b][i]
  if (live && tid < n * n) {
    dfl xv[n];
#pragma unroll
    for (int a = 0; a < n; ++a) xv[a] = sX[tid * L::XL + a];
    if constexpr (EO) {
      df2 xpm[n / 2];
      dfl yb[Q], yg[Q];
      eo_split2<n>(xv, xpm);
      eo_apply2<EB, 1>(xpm, xv[n / 2], yb);
      if (DIFF) eo_apply2<EG, -1>(xpm, xv[n / 2], yg);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        S1[tid * DQ1 + i] = yb[i];
        if (DIFF) S1[L::S1C + tid * DQ1 + i] = yg[i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        dfl sb = df_zero(), sg = df_zero();
#pragma unroll
        for (int a = 0; a < n; ++a) {
          df_fma(sb, T::B(i, a), xv[a]);
          if (DIFF) df_fma(sg, T::G(i, a), xv[a]);
        }
        S1[tid * DQ1 + i] = df_norm(sb);
        if (DIFF) S1[L::S1C + tid * DQ1 + i] = df_norm(sg);
      }
    }
  }
  __syncthreads();

  // stage 2 (y): line (i,c) -> S2[m][c][j][i]
  if (live && tid < Q * n) {
    const int i = tid % Q, c = tid / Q;
    dfl vb[n], vg[n];
#pragma unroll
    for (int b = 0; b < n; ++b) {
      vb[b] = S1[(b + n * c) * DQ1 + i];
      if (DIFF) vg[b] = S1[L::S1C + (b + n * c) * DQ1 + i];
    }
    if constexpr (EO) {
      df2 bpm[n / 2];
      dfl yb[Q];
      eo_split2<n>(vb, bpm);
      eo_apply2<EB, 1>(bpm, vb[n / 2], yb);
#pragma unroll
      for (int j = 0; j < Q; ++j) S2[(DIFF ? 2 * L::S2C : 0) + c * L::P2 + j * Q + i] = yb[j];
      if (DIFF) {
        dfl yg[Q];
        eo_apply2<EG, -1>(bpm, vb[n / 2], yg);
#pragma unroll
        for (int j = 0; j < Q; ++j) S2[L::S2C + c * L::P2 + j * Q + i] = yg[j];
        df2 gpm[n / 2];
        eo_split2<n>(vg, gpm);
        eo_apply2<EB, 1>(gpm, vg[n / 2], yg);
#pragma unroll
        for (int j = 0; j < Q; ++j) S2[c * L::P2 + j * Q + i] = yg[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        dfl bb = df_zero(), bg = df_zero(), gb = df_zero();
#pragma unroll
        for (int b = 0; b < n; ++b) {
          df_fma(bb, T::B(j, b), vb[b]);
          if (DIFF) {
            df_fma(bg, T::G(j, b), vb[b]);
            df_fma(gb, T::B(j, b), vg[b]);
          }
        }
        const int o = c * L::P2 + j * Q + i;
        if (DIFF) {
          S2[o] = df_norm(gb);
          S2[L::S2C + o] = df_norm(bg);
          S2[2 * L::S2C + o] = df_norm(bb);
        } else {
          S2[o] = df_norm(bb);
        }
      }
    }
  }
  __syncthreads();

  // stage 3 (z) + D + stage 3^T per (i,j) column, in registers
  if (live) {
    dfl c0[n], c1[n], c2[n], a0[n], a1[n], a2[n];
#pragma unroll
    for (int c = 0; c < n; ++c) {
      c0[c] = S2[c * L::P2 + tid];
      if (DIFF) {
        c1[c] = S2[L::S2C + c * L::P2 + tid];
        c2[c] = S2[2 * L::S2C + c * L::P2 + tid];
      }
      a0[c] = df_zero();
      if (DIFF) a1[c] = a2[c] = df_zero();
    }
    const float2* dE = qd + (e0 + el) * (L::NC * L::Q3) + tid;
    // (loading D one point ahead was measured 1-8 % slower here: this kernel is bound by
    // arithmetic and the registers are better spent on it)
    if constexpr (EO && DfTune<P, Q, DIFF>::EO3) {
      // z contraction, D and z^T in even/odd form over the mirrored point pairs (k, Q-1-k):
      // u at both points from the split column, then the pair's sums and differences of v
      // accumulate into the even (E) and odd (O) halves of a (mirrored outputs recombined
      // at the end)
      constexpr int HN = n / 2, HQ = Q / 2;
      // packed pairs: (c+, c-) of the column, (E, O) of the z contraction, (p, q) of v at the
      // point pair, (a_E, a_O) of the transposed contraction; D of both points as pairs
      df2 cpm0[HN], cpm1[HN], cpm2[HN], aeo0[HN], aeo1[HN], aeo2[HN];
      dfl am0 = df_zero(), am1 = df_zero(), am2 = df_zero();
      eo_split2<n>(c0, cpm0);
      if (DIFF) {
        eo_split2<n>(c1, cpm1);
        eo_split2<n>(c2, cpm2);
      }
#pragma unroll
      for (int c = 0; c < HN; ++c) {
        aeo0[c] = df2_zero();
        if (DIFF) aeo1[c] = aeo2[c] = df2_zero();
      }
      // v = D u at one point k (the middle point of an odd Q), scalar
      auto dpoint = [&](int k, dfl u0, dfl u1, dfl u2, dfl& v0, dfl& v1, dfl& v2) {
        float2 dc[L::NC];
#pragma unroll
        for (int m = 0; m < L::NC; ++m) dc[m] = __ldg(dE + k * Q * Q + m * L::Q3);
        if (DIFF) {
          const int i1 = 1 % L::NC, i2 = 2 % L::NC, i3 = 3 % L::NC, i4 = 4 % L::NC, i5 = 5 % L::NC;
          const dfl d00 = {dc[0].x, dc[0].y}, d01 = {dc[i1].x, dc[i1].y}, d02 = {dc[i2].x, dc[i2].y},
                    d11 = {dc[i3].x, dc[i3].y}, d12 = {dc[i4].x, dc[i4].y}, d22 = {dc[i5].x, dc[i5].y};
          v0 = df_zero(); v1 = df_zero(); v2 = df_zero();
          df_fma(v0, d00, u0);
          df_fma(v0, d01, u1);
          df_fma(v0, d02, u2);
          df_fma(v1, d01, u0);
          df_fma(v1, d11, u1);
          df_fma(v1, d12, u2);
          df_fma(v2, d02, u0);
          df_fma(v2, d12, u1);
          df_fma(v2, d22, u2);
          v0 = df_norm(v0);
          v1 = df_norm(v1);
          v2 = df_norm(v2);
        } else {
          v0 = df_zero();
          df_fma(v0, dfl{dc[0].x, dc[0].y}, u0);
          v0 = df_norm(v0);
        }
      };
#pragma unroll KU
      for (int kk = 0; kk < HQ; ++kk) {
        const int k2 = Q - 1 - kk;
        df2 eo0 = df2_zero(), eo1 = df2_zero(), eo2 = df2_zero();  // (E, O)
#pragma unroll
        for (int i = 0; i < HN; ++i) {
          df2_fma(eo0, EB::EDh(kk, i), EB::EDl(kk, i), cpm0[i].h, cpm0[i].l);
          if (DIFF) {
            df2_fma(eo1, EB::EDh(kk, i), EB::EDl(kk, i), cpm1[i].h, cpm1[i].l);
            df2_fma(eo2, EG::EDh(kk, i), EG::EDl(kk, i), cpm2[i].h, cpm2[i].l);
          }
        }
        dfl e0 = df2_x(eo0), e1 = df2_x(eo1), e2 = df2_x(eo2);
        if (n % 2) {
          df_fma(e0, EB::MC(kk), c0[HN]);
          if (DIFF) {
            df_fma(e1, EB::MC(kk), c1[HN]);
            df_fma(e2, EG::MC(kk), c2[HN]);
          }
        }
        // u at (kk, k2): (E + O, E - O); the G component's mirror is O - E
        const df2 u0 = df2_sumdiff(e0, df2_y(eo0));
        df2 u1 = u0, u2 = u0;
        if (DIFF) {
          u1 = df2_sumdiff(e1, df2_y(eo1));
          u2 = df2_sumdiff(e2, df2_y(eo2));
          u2.h.y = -u2.h.y;
          u2.l.y = -u2.l.y;
        }
        df2 v0, v1, v2;
        df2_dpoint<DIFF, L::NC, Q * Q, L::Q3>(dE, kk, k2, u0, u1, u2, v0, v1, v2);
        // (p, q) = (v(kk) + v(k2), v(kk) - v(k2))
        const df2 pq0 = df2_sumdiff(df2_x(v0), df2_y(v0));
        df2 pq1 = pq0, pq2 = pq0;
        if (DIFF) {
          pq1 = df2_sumdiff(df2_x(v1), df2_y(v1));
          pq2 = df2_sumdiff(df2_x(v2), df2_y(v2));
        }
#pragma unroll
        for (int c = 0; c < HN; ++c) {
          df2_fma(aeo0[c], EBT::EDh(c, kk), EBT::EDl(c, kk), pq0.h, pq0.l);
          if (DIFF) {
            df2_fma(aeo1[c], EBT::EDh(c, kk), EBT::EDl(c, kk), pq1.h, pq1.l);
            df2_fma(aeo2[c], EGT::EDh(c, kk), EGT::EDl(c, kk), pq2.h, pq2.l);
          }
        }
        if (n % 2) {
          df_fma(am0, EBT::MR(kk), df2_x(pq0));
          if (DIFF) {
            df_fma(am1, EBT::MR(kk), df2_x(pq1));
            df_fma(am2, EGT::MR(kk), df2_y(pq2));
          }
        }
      }
      if (Q % 2) {  // the middle point
        dfl u0 = df_zero(), u1 = df_zero(), u2 = df_zero();
#pragma unroll
        for (int i = 0; i < HN; ++i) {
          df_fma(u0, EB::MR(i), df2_x(cpm0[i]));
          if (DIFF) {
            df_fma(u1, EB::MR(i), df2_x(cpm1[i]));
            df_fma(u2, EG::MR(i), df2_y(cpm2[i]));
          }
        }
        if (n % 2) {
          df_fma(u0, EB::MR(HN), c0[HN]);
          if (DIFF) df_fma(u1, EB::MR(HN), c1[HN]);
        }
        dfl v0, v1, v2;
        dpoint(HQ, df_norm(u0), df_norm(u1), df_norm(u2), v0, v1, v2);
#pragma unroll
        for (int c = 0; c < HN; ++c) {
          dfl t0 = df2_x(aeo0[c]);
          df_fma(t0, EBT::MC(c), v0);
          aeo0[c].h.x = t0.h;
          aeo0[c].l.x = t0.l;
          if (DIFF) {
            dfl t1 = df2_x(aeo1[c]), t2 = df2_x(aeo2[c]);
            df_fma(t1, EBT::MC(c), v1);
            df_fma(t2, EGT::MC(c), v2);
            aeo1[c].h.x = t1.h;
            aeo1[c].l.x = t1.l;
            aeo2[c].h.x = t2.h;
            aeo2[c].l.x = t2.l;
          }
        }
        if (n % 2) {
          df_fma(am0, EBT::MR(HQ), v0);
          if (DIFF) df_fma(am1, EBT::MR(HQ), v1);
        }
      }
#pragma unroll
      for (int c = 0; c < HN; ++c) {
        const df2 r0 = df2_sumdiff(df2_x(aeo0[c]), df2_y(aeo0[c]));
        a0[c] = df2_x(r0);
        a0[n - 1 - c] = df2_y(r0);
        if (DIFF) {
          const df2 r1 = df2_sumdiff(df2_x(aeo1[c]), df2_y(aeo1[c]));
          const df2 r2 = df2_sumdiff(df2_x(aeo2[c]), df2_y(aeo2[c]));
          a1[c] = df2_x(r1);
          a1[n - 1 - c] = df2_y(r1);
          a2[c] = df2_x(r2);
          a2[n - 1 - c] = df_neg(df2_y(r2));
        }
      }
      if (n % 2) {
        a0[HN] = am0;
        if (DIFF) {
          a1[HN] = am1;
          a2[HN] = am2;
        }
      }
    } else if constexpr (!DfTune<P, Q, DIFF>::PK3) {
#pragma unroll KU
    for (int k = 0; k < Q; ++k) {
      float2 dc[L::NC];
#pragma unroll
      for (int m = 0; m < L::NC; ++m) dc[m] = __ldg(dE + k * Q * Q + m * L::Q3);
      if (DIFF) {
        dfl u0 = df_zero(), u1 = df_zero(), u2 = df_zero();
#pragma unroll
        for (int c = 0; c < n; ++c) {
          df_fma(u0, T::B(k, c), c0[c]);
          df_fma(u1, T::B(k, c), c1[c]);
          df_fma(u2, T::G(k, c), c2[c]);
        }
        u0 = df_norm(u0);
        u1 = df_norm(u1);
        u2 = df_norm(u2);
        const int i1 = 1 % L::NC, i2 = 2 % L::NC, i3 = 3 % L::NC, i4 = 4 % L::NC, i5 = 5 % L::NC;
        const dfl d00 = {dc[0].x, dc[0].y}, d01 = {dc[i1].x, dc[i1].y}, d02 = {dc[i2].x, dc[i2].y},
                  d11 = {dc[i3].x, dc[i3].y}, d12 = {dc[i4].x, dc[i4].y}, d22 = {dc[i5].x, dc[i5].y};
        dfl v0 = df_zero(), v1 = df_zero(), v2 = df_zero();
        df_fma(v0, d00, u0);
        df_fma(v0, d01, u1);
        df_fma(v0, d02, u2);
        df_fma(v1, d01, u0);
        df_fma(v1, d11, u1);
        df_fma(v1, d12, u2);
        df_fma(v2, d02, u0);
        df_fma(v2, d12, u1);
        df_fma(v2, d22, u2);
        v0 = df_norm(v0);
        v1 = df_norm(v1);
        v2 = df_norm(v2);
#pragma unroll
        for (int c = 0; c < n; ++c) {
          df_fma(a0[c], T::B(k, c), v0);
          df_fma(a1[c], T::B(k, c), v1);
          df_fma(a2[c], T::G(k, c), v2);
        }
      } else {
        dfl u = df_zero();
#pragma unroll
        for (int c = 0; c < n; ++c) df_fma(u, T::B(k, c), c0[c]);
        u = df_norm(u);
        dfl v = df_zero();
        df_fma(v, dfl{dc[0].x, dc[0].y}, u);
        v = df_norm(v);
#pragma unroll
        for (int c = 0; c < n; ++c) df_fma(a0[c], T::B(k, c), v);
      }
    }
    } else {
      // direct form in packed pairs: the quadrature points (2kp, 2kp+1) of the forward
      // contractions (row pairs of the tables, input broadcast), D at both points, and the
      // transposed contraction over column pairs (c, c+1) (output broadcast); per output the
      // scalar steps, in the same order
      constexpr int QH = (Q + 1) / 2, NP = n / 2;
      constexpr bool ODDN = (n % 2) != 0;
      df2 A0[NP], A1[NP], A2[NP];
      dfl z0 = df_zero(), z1 = df_zero(), z2 = df_zero();  // column n - 1 of an odd n
#pragma unroll
      for (int cp = 0; cp < NP; ++cp) {
        A0[cp] = df2_zero();
        if (DIFF) A1[cp] = A2[cp] = df2_zero();
      }
#pragma unroll KU
      for (int kp = 0; kp < QH; ++kp) {
        const int ka = 2 * kp, kb = (2 * kp + 1 < Q) ? 2 * kp + 1 : 2 * kp;  // (an odd Q's last pair repeats its point)
        df2 U0 = df2_zero(), U1 = df2_zero(), U2 = df2_zero();
#pragma unroll
        for (int c = 0; c < n; ++c) {
          df2_fma(U0, T::Brh(kp, c), T::Brl(kp, c), bcast2(c0[c].h), bcast2(c0[c].l));
          if (DIFF) {
            df2_fma(U1, T::Brh(kp, c), T::Brl(kp, c), bcast2(c1[c].h), bcast2(c1[c].l));
            df2_fma(U2, T::Grh(kp, c), T::Grl(kp, c), bcast2(c2[c].h), bcast2(c2[c].l));
          }
        }
        U0 = df2_norm(U0);
        if (DIFF) {
          U1 = df2_norm(U1);
          U2 = df2_norm(U2);
        }
        df2 V0, V1, V2;
        df2_dpoint<DIFF, L::NC, Q * Q, L::Q3>(dE, ka, kb, U0, U1, U2, V0, V1, V2);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = 2 * kp + h;
          if (k >= Q) break;
          const dfl v0 = h ? df2_y(V0) : df2_x(V0);
#pragma unroll
          for (int cp = 0; cp < NP; ++cp) {
            df2_fma(A0[cp], T::Bch(k, cp), T::Bcl(k, cp), bcast2(v0.h), bcast2(v0.l));
            if (DIFF) {
              const dfl v1 = h ? df2_y(V1) : df2_x(V1), v2 = h ? df2_y(V2) : df2_x(V2);
              df2_fma(A1[cp], T::Bch(k, cp), T::Bcl(k, cp), bcast2(v1.h), bcast2(v1.l));
              df2_fma(A2[cp], T::Gch(k, cp), T::Gcl(k, cp), bcast2(v2.h), bcast2(v2.l));
            }
          }
          if (ODDN) {
            df_fma(z0, dfl{T::Bch(k, NP).x, T::Bcl(k, NP).x}, v0);
            if (DIFF) {
              df_fma(z1, dfl{T::Bch(k, NP).x, T::Bcl(k, NP).x}, h ? df2_y(V1) : df2_x(V1));
              df_fma(z2, dfl{T::Gch(k, NP).x, T::Gcl(k, NP).x}, h ? df2_y(V2) : df2_x(V2));
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < n; ++c) {
        const bool last = ODDN && c == n - 1;
        const int cp = last ? 0 : c / 2;
        a0[c] = last ? z0 : ((c & 1) ? df2_y(A0[cp]) : df2_x(A0[cp]));
        if (DIFF) {
          a1[c] = last ? z1 : ((c & 1) ? df2_y(A1[cp]) : df2_x(A1[cp]));
          a2[c] = last ? z2 : ((c & 1) ? df2_y(A2[cp]) : df2_x(A2[cp]));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < n; ++c) {
      S2[c * L::P2 + tid] = df_norm(a0[c]);
      if (DIFF) {
        S2[L::S2C + c * L::P2 + tid] = df_norm(a1[c]);
        S2[2 * L::S2C + c * L::P2 + tid] = df_norm(a2[c]);
      }
    }
  }
  __syncthreads();

  // stage 2^T (y)
  if (live && tid < Q * n) {
    const int i = tid % Q, c = tid / Q;
    dfl v0[Q], v1[Q], v2[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      v0[j] = S2[c * L::P2 + j * Q + i];
      if (DIFF) {
        v1[j] = S2[L::S2C + c * L::P2 + j * Q + i];
        v2[j] = S2[2 * L::S2C + c * L::P2 + j * Q + i];
      }
    }
    if constexpr (EO) {
      df2 pm0[Q / 2];
      dfl y0[n];
      eo_split2<Q>(v0, pm0);
      eo_apply2<EBT, 1>(pm0, v0[Q / 2], y0);
#pragma unroll
      for (int b = 0; b < n; ++b) S1[(b + n * c) * DQ1 + i] = y0[b];
      if (DIFF) {
        df2 pm1[Q / 2];
        dfl y1[n];
        eo_split2<Q>(v1, pm1);
        eo_apply2<EGT, -1>(pm1, v1[Q / 2], y1);
        eo_split2<Q>(v2, pm0);
        eo_apply2<EBT, 1>(pm0, v2[Q / 2], y0);
#pragma unroll
        for (int b = 0; b < n; ++b) S1[L::S1C + (b + n * c) * DQ1 + i] = df_add(y1[b], y0[b]);
      }
    } else {
#pragma unroll
      for (int b = 0; b < n; ++b) {
        dfl t0 = df_zero(), t1 = df_zero();
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          df_fma(t0, T::B(j, b), v0[j]);
          if (DIFF) {
            df_fma(t1, T::G(j, b), v1[j]);
            df_fma(t1, T::B(j, b), v2[j]);
          }
        }
        S1[(b + n * c) * DQ1 + i] = df_norm(t0);
        if (DIFF) S1[L::S1C + (b + n * c) * DQ1 + i] = df_norm(t1);
      }
    }
  }
  __syncthreads();

  // stage 1^T (x) and G^T (FP64 atomics)
  if (live && tid < n * n) {
    dfl t0[Q], t1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      t0[i] = S1[tid * DQ1 + i];
      if (DIFF) t1[i] = S1[L::S1C + tid * DQ1 + i];
    }
    dfl ys[n];
    if constexpr (EO) {
      df2 ppm[Q / 2];
      dfl yb[n];
      if (DIFF) {
        eo_split2<Q>(t0, ppm);
        eo_apply2<EGT, -1>(ppm, t0[Q / 2], ys);
        eo_split2<Q>(t1, ppm);
        eo_apply2<EBT, 1>(ppm, t1[Q / 2], yb);
#pragma unroll
        for (int a = 0; a < n; ++a) ys[a] = df_add(ys[a], yb[a]);
      } else {
        eo_split2<Q>(t0, ppm);
        eo_apply2<EBT, 1>(ppm, t0[Q / 2], ys);
      }
    } else {
#pragma unroll
      for (int a = 0; a < n; ++a) {
        dfl s = df_zero();
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (DIFF) {
            df_fma(s, T::G(i, a), t0[i]);
            df_fma(s, T::B(i, a), t1[i]);
          } else {
            df_fma(s, T::B(i, a), t0[i]);
          }
        }
        ys[a] = s;
      }
    }
#pragma unroll
    for (int a = 0; a < n; ++a) {
      const dfl s = ys[a];
      const int gi = g[a + n * tid];
      if (gi >= 0) {
        atomicAdd(y + gi, rescaled ? df_to(s) * yscale : df_to(s));
      } else if (!((~gi) & ESS_SKIP)) {
        atomicAdd(y + (~gi), x[~gi]);
      }
    }
  }
}

// (MINB scales with NE_DIV: half-size blocks keep the register cap of the full-size ones)
template <int P, int Q, bool DIFF, int NE_DIV = 1, int MINB = DfTune<P, Q, DIFF>::MINB * NE_DIV,
          int KU = DfTune<P, Q, DIFF>::KU, int PF = 2>
__global__ void __launch_bounds__(DfShape<P, Q, DIFF, NE_DIV>::TPE * DfShape<P, Q, DIFF, NE_DIV>::NE, MINB)
pa_apply_df(int E, const int* __restrict__ gmap, const float2* __restrict__ qd, const double* __restrict__ x,
            double* __restrict__ y, const int* __restrict__ skip, const int* __restrict__ elem_prob,
            const int* __restrict__ prob_done, int dexp) {
  constexpr int NE = DfShape<P, Q, DIFF, NE_DIV>::NE;
  if (skip && *skip) return;
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  df_tile<P, Q, DIFF, KU, PF, NE_DIV>(e0, (int)((E - e0) < NE ? (E - e0) : NE), gmap, qd, x, y, elem_prob, prob_done,
                                      dexp);
}

// Persistent form over a work list (the batch's iteration loop), as pa_apply_f32_tiles
template <int P, int Q, bool DIFF, int NE_DIV = 1, int MINB = DfTune<P, Q, DIFF>::MINB * NE_DIV>
__global__ void __launch_bounds__(DfShape<P, Q, DIFF, NE_DIV>::TPE * DfShape<P, Q, DIFF, NE_DIV>::NE, MINB)
pa_apply_df_tiles(const int2* __restrict__ tiles, const int* __restrict__ act, const int* __restrict__ nact,
                  const int* __restrict__ gmap, const float2* __restrict__ qd, const double* __restrict__ x,
                  double* __restrict__ y, const int* __restrict__ skip, int dexp) {
  if (skip && *skip) return;
  const int count = *nact;
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const int2 tl = tiles[act[i]];
    df_tile<P, Q, DIFF, DfTune<P, Q, DIFF>::KU, 2, NE_DIV>(tl.x, tl.y, gmap, qd, x, y, nullptr, nullptr, dexp);
    __syncthreads();  // (the next tile reuses the shared buffers)
  }
}

// FP64 D -> (hi, lo) float pairs, same layout [e][comp][q^3]
__global__ void split_to_df(int64_t count, const double* __restrict__ qd, float2* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const dfl v = df_from(qd[t]);
    out[t] = make_float2(v.h, v.l);
  }
}

}  // namespace fepa

namespace fepa {

// ---------------------------------------------------------------------------
// diag(A) in double-float (the matrix-free diagonal of Sec. 2.1 by sum factorisation):
// diag(a,b,c) = sum_m wt_m sum_{i,j,k} X_m[i][a] Y_m[j][b] Z_m[k][c] D_m(i,j,k), the
// 1D tables being products B B, B G or G G per direction and component (mass: B B in
// every direction).  Same stages as the FP64 kernel (z in registers, then y and x
// through shared memory), several elements per block, D read as (hi, lo) pairs.
// ---------------------------------------------------------------------------
template <int P, int Q, bool DIFF>
struct DiagDfShape {
  static constexpr int N = P + 1, NC = DIFF ? 6 : 1, TPE = Q * Q;
  static constexpr int PER = NC * N * Q * Q + NC * N * N * Q;  // T1 + T2 values per element
  static constexpr int NE0 = (256 / TPE) > 0 ? (256 / TPE) : 1;
  static constexpr int NE = (NE0 * PER * 8 > 160 * 1024) ? ((160 * 1024) / (PER * 8) > 0 ? (160 * 1024) / (PER * 8) : 1)
                                                          : NE0;
  static constexpr int SMEM = (3 * Q * N + NE * PER) * 8;
};

template <int P, int Q, bool DIFF>
__global__ void __launch_bounds__(DiagDfShape<P, Q, DIFF>::TPE * DiagDfShape<P, Q, DIFF>::NE)
pa_diag_df(int E, const int* __restrict__ gmap, const float2* __restrict__ qd, double* __restrict__ diag) {
  using S = DiagDfShape<P, Q, DIFF>;
  using T = TabDf<P, Q>;
  constexpr int n = S::N, NC = S::NC, TPE = S::TPE, NE = S::NE, Q3 = Q * Q * Q;
  extern __shared__ __align__(16) unsigned char smem_dg[];
  dfl* tab = reinterpret_cast<dfl*>(smem_dg);  // [3][Q][n]: B B, B G, G G
  const int tid = threadIdx.x, el = threadIdx.y, flat = el * TPE + tid;
  for (int l = flat; l < Q * n; l += TPE * NE) {
    const int i = l / n, a = l - i * n;
    const dfl b = T::B(i, a), g = T::G(i, a);
    tab[l] = df_mul(b, b);
    tab[Q * n + l] = df_mul(b, g);
    tab[2 * Q * n + l] = df_mul(g, g);
  }
  dfl* T1 = tab + 3 * Q * n + el * S::PER;  // [m][c][j][i]
  dfl* T2 = T1 + NC * n * TPE;              // [m][c][b][i]
  const int64_t e = (int64_t)blockIdx.x * NE + el;
  const bool live = e < E;
  __syncthreads();
  // table per direction and component (xx, xy, xz, yy, yz, zz): 0 BB, 1 BG, 2 GG
  constexpr int selx[6] = {2, 1, 1, 0, 0, 0}, sely[6] = {0, 1, 0, 2, 1, 0}, selz[6] = {0, 0, 1, 0, 1, 2};
  if (live) {  // z
    const float2* de = qd + e * NC * Q3 + tid;
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const dfl* Z = tab + (DIFF ? selz[m] : 0) * Q * n;
      dfl acc[n];
#pragma unroll
      for (int c = 0; c < n; ++c) acc[c] = df_zero();
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const dfl dv = df_ld(de + m * Q3 + k * TPE);
#pragma unroll
        for (int c = 0; c < n; ++c) df_fma(acc[c], dv, Z[k * n + c]);
      }
#pragma unroll
      for (int c = 0; c < n; ++c) T1[(m * n + c) * TPE + tid] = df_norm(acc[c]);
    }
  }
  __syncthreads();
  if (live)  // y
    for (int w = tid; w < NC * n * n * Q; w += TPE) {
      const int i = w % Q, b = (w / Q) % n, mc = w / (n * Q), m = mc / n;
      const dfl* Y = tab + (DIFF ? sely[m] : 0) * Q * n;
      const dfl* src = T1 + mc * TPE + i;
      dfl s = df_zero();
#pragma unroll
      for (int j = 0; j < Q; ++j) df_fma(s, src[j * Q], Y[j * n + b]);
      T2[w] = df_norm(s);
    }
  __syncthreads();
  if (live) {  // x, weights, scatter
    const int* g = gmap + e * (n * n * n);
    for (int w = tid; w < n * n * n; w += TPE) {
      const int a = w % n, cb = w / n;
      dfl s = df_zero();
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        const dfl* X = tab + (DIFF ? selx[m] : 0) * Q * n;
        const dfl* src = T2 + (m * n * n + cb) * Q;
        dfl sm = df_zero();
#pragma unroll
        for (int i = 0; i < Q; ++i) df_fma(sm, src[i], X[i * n + a]);
        sm = df_norm(sm);
        if (DIFF && (m == 1 || m == 2 || m == 4)) sm = dfl{2.f * sm.h, 2.f * sm.l};  // off-diagonal components
        s = df_add(s, sm);
      }
      const int gi = g[w];
      if (gi >= 0)
        atomicAdd(diag + gi, df_to(s));
      else if (!((~gi) & ESS_SKIP))
        atomicAdd(diag + (~gi), 1.0);
    }
  }
}

}  // namespace fepa
