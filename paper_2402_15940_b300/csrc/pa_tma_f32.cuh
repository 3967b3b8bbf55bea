// FP32 fused partial-assembly action for the mixed-precision solve (the operator
// y = G^T B^T D B G x of Fig. fig_feod, arXiv 2402.15940), built for an HBM-bound
// kernel on sm_103a.  Common to all variants:
//   * the 1D tables live in __constant__ memory at compile-time offsets, so with the
//     loops unrolled they are free FMA operands -- as pairs of entries, so that one packed
//     FMA (two FP32 FMAs in one instruction) produces two outputs of a line;
//   * every stage is register-blocked: a thread loads one line of its element once
//     and produces all outputs of that line; stage 3, the pointwise D and the
//     transposed stage 3 stay in registers per (i,j) column;
//   * shared-memory line and plane strides are padded to spread banks.
// Variants (chosen per (p, q, form) by the autotuner in fepa.cu):
//   0  one element group per block, the group's D staged by one TMA bulk copy
//      (cp.async.bulk + mbarrier) that overlaps the gather and stages 1-2;
//   1  as 0 with D read straight from HBM in stage 3 (smaller footprint, more warps);
//   2  as 1 with half as many elements per block;
//   3  persistent blocks, software-pipelined over element groups: while group g is
//      computed, D(g+1) arrives by TMA, the map of g+1 is loaded into registers and
//      x(g+1) is gathered by cp.async (asynchronous 4-byte copies) into the other
//      buffer, so the dependent map -> x -> compute latency chain is hidden.
// D here is the FP32 copy with each component padded to a multiple of 4 floats, so
// every element's block is a multiple of 16 bytes (the bulk-copy granularity).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "cg_kernels.cuh"
#include "pa_kernels.cuh"

namespace fepa {

// FP32 1D tables of every compiled (P, Q) as float2 pairs, for the packed FMA (__ffma2_rn:
// two FMAs in one instruction, each component rounded as fmaf), with a table pair as one
// constant-bank operand and the other operand a pair or a broadcast scalar:
//   rows     R[kp][a] = (T(2kp, a), T(2kp+1, a)),  kp < ceil(Q/2)  (.y = 0 past row Q-1)
//   columns  C[k][ap] = (T(k, 2ap), T(k, 2ap+1)),  ap < ceil(n/2)  (.y = 0 past column n-1)
// for T = B, G (Q x n, T(i, a) = basis a or its derivative at point i); slots packed in the
// order (1, 2), (1, 3), (2, 3), (2, 4), ... (8, 10).
constexpr int tab32_slot_pairs(int P, int Q) { return 2 * (((Q + 1) / 2) * (P + 1) + Q * ((P + 2) / 2)); }
constexpr int tab32_offset(int P, int Q) {
  int off = 0;
  for (int p = 1; p <= 8; ++p)
    for (int q = p + 1; q <= p + 2; ++q) {
      if (p == P && q == Q) return off;
      off += tab32_slot_pairs(p, q);
    }
  return off;  // past the last slot: the total
}
constexpr int TAB32_PAIRS = tab32_offset(9, 0);
__constant__ float2 c_tab32[TAB32_PAIRS];

template <int P, int Q>
struct Tab32 {
  static_assert(Q == P + 1 || Q == P + 2, "compiled q");
  static constexpr int N = P + 1, QH = (Q + 1) / 2, NH = (N + 1) / 2;
  static constexpr int BR = tab32_offset(P, Q), GR = BR + QH * N, BC = GR + QH * N, GC = BC + Q * NH;
  static __device__ __forceinline__ float2 Br(int kp, int a) { return c_tab32[BR + kp * N + a]; }
  static __device__ __forceinline__ float2 Gr(int kp, int a) { return c_tab32[GR + kp * N + a]; }
  static __device__ __forceinline__ float2 Bc(int k, int ap) { return c_tab32[BC + k * NH + ap]; }
  static __device__ __forceinline__ float2 Gc(int k, int ap) { return c_tab32[GC + k * NH + ap]; }
  static __device__ __forceinline__ float B(int i, int a) { return (i & 1) ? Br(i >> 1, a).y : Br(i >> 1, a).x; }
  static __device__ __forceinline__ float G(int i, int a) { return (i & 1) ? Gr(i >> 1, a).y : Gr(i >> 1, a).x; }
};

// the pair tables of (p, q) from the row-major q x n tables B, G (host)
inline std::vector<float2> tab32_pairs(int p, int q, const std::vector<float>& B, const std::vector<float>& G) {
  const int n = p + 1, qh = (q + 1) / 2, nh = (n + 1) / 2;
  std::vector<float2> out;
  out.reserve(tab32_slot_pairs(p, q));
  for (const std::vector<float>* T : {&B, &G})
    for (int kp = 0; kp < qh; ++kp)
      for (int a = 0; a < n; ++a)
        out.push_back(make_float2((*T)[2 * kp * n + a], 2 * kp + 1 < q ? (*T)[(2 * kp + 1) * n + a] : 0.f));
  for (const std::vector<float>* T : {&B, &G})
    for (int k = 0; k < q; ++k)
      for (int ap = 0; ap < nh; ++ap)
        out.push_back(make_float2((*T)[k * n + 2 * ap], 2 * ap + 1 < n ? (*T)[k * n + 2 * ap + 1] : 0.f));
  return out;
}

// upload the FP32 pair tables of (p, q) into their constant-memory slot
inline cudaError_t upload_tab32(int p, int q, const std::vector<float>& B, const std::vector<float>& G,
                                cudaStream_t s) {
  const std::vector<float2> t = tab32_pairs(p, q, B, G);
  return cudaMemcpyToSymbolAsync(c_tab32, t.data(), t.size() * sizeof(float2), tab32_offset(p, q) * sizeof(float2),
                                 cudaMemcpyHostToDevice, s);
}

__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }

// Which stages of the FP32 action use the packed FMA, per (P, Q, form): bit 0 stage 1,
// bit 1 stage 2, bit 2 stage 3 (points paired; else one point at a time, in scalar FMAs),
// bit 3 stage 3's transposed contraction (with bit 2 clear), bit 4 stage 2^T, bit 5 stage 1^T.
// Measured on B300 (variants 1 and 2 against the all-scalar build, stand-alone launches):
// all stages packed is 5-29 % faster from p = 5 and for mass at p = 4, 8; where pairing the
// points of stage 3 costs registers (and resident blocks) it stays scalar or pairs only its
// transposed contraction: diffusion p = 4, q = 6 2 % faster (all packed: 48 registers, 5 %
// slower), p = 8 23 %, p = 1-3 within 1 %.
constexpr int pack32_mask(int P, int Q, bool DIFF) {
  return DIFF ? ((Q == P + 2 && P == 4) ? 51 : (Q == P + 2 && (P <= 3 || P == 8)) ? 59 : 63)
              : (P == 7 ? 51 : 63);
}
template <int P, int Q, bool DIFF>
struct Pack32 {
  static constexpr int MASK = pack32_mask(P, Q, DIFF);
  static constexpr bool S1 = MASK & 1, S2 = MASK & 2, S3F = MASK & 4, S3T = (MASK & 4) || (MASK & 8),
                        S2T = MASK & 16, S1T = MASK & 32;
};

// S1 strides and element padding per (P, Q) of the double-float kernel's layout (the FP32
// kernels use F32Smem below), from an exhaustive search of a model of the warp access
// patterns (stage 1 writing and stage 1^T reading line (b,c); stage 2 reading and stage
// 2^T writing along b for thread (i,c); elements dealt over the block): the
// fewest shared-memory wavefronts, 27-50 % fewer than the plain odd strides.  Measured on
// B300: 7-11 % faster for p = 2, 3, neutral at p = 4, 4-13 % slower from p = 5 (where the
// model's pick changes more than the conflicts), so used up to p = 4.
struct S1Pick {
  int q1, cs, pad;
};
constexpr S1Pick s1_pick(int P, int Q) {
  return (P == 1 && Q == 3)   ? S1Pick{8, 16, 1}
         : (P == 2 && Q == 3) ? S1Pick{5, 35, 28}
         : (P == 2 && Q == 4) ? S1Pick{5, 20, 0}
         : (P == 3 && Q == 5) ? S1Pick{8, 37, 16}
         : (P == 4 && Q == 5) ? S1Pick{7, 37, 28}
         : (P == 4 && Q == 6) ? S1Pick{9, 45, 5}
                              : S1Pick{Q | 1, (P + 1) * (Q | 1), 0};
}

// Shared-memory layout of one element's stage buffers of the double-float kernel (in
// elements of its word type), padded:
//   X  [c][b][a]     line (b,c) of length n at stride XL (odd)
//   S1 [m][c][b][i]  entry (b,c,i) at b*Q1 + c*CS + i (strides from s1_pick)
//   S2 [m][c][j][i]  plane c of Q*Q at stride P2 (P2 = Q mod 32: consecutive planes
//                    start Q banks apart)
// (the double-float kernel takes these sizes with its own line stride Q1 in S1)
template <int P, int Q, bool DIFF>
struct F32Layout {
  static constexpr int N = P + 1;
  static constexpr int NC = DIFF ? 6 : 1;
  static constexpr int Q3 = Q * Q * Q;
  static constexpr int DSTRIDE = (Q3 + 3) & ~3;  // floats per stored D component (16-byte multiple)
  static constexpr int DELEM = NC * DSTRIDE;     // floats of D per element
  static constexpr int NC1 = DIFF ? 2 : 1;
  static constexpr int NC2 = DIFF ? 3 : 1;
  static constexpr int XL = N | 1;
  static constexpr int Q1 = s1_pick(P, Q).q1;
  static constexpr int CS = s1_pick(P, Q).cs;  // >= N * Q1
  static constexpr int P2 = Q * Q + (((Q - (Q * Q) % 32) % 32) + 32) % 32;
  static constexpr int XSZ = XL * N * N;
  static constexpr int S1C = CS * N;      // one S1 component
  static constexpr int S2C = P2 * N;      // one S2 component
  static constexpr int WORK = NC1 * S1C + NC2 * S2C + s1_pick(P, Q).pad;
  static_assert(CS >= N * Q1 && Q1 >= Q, "S1 strides");
  static constexpr int TPE = Q * Q;
  static constexpr int NE0 = (256 / TPE) > 0 ? (256 / TPE) : 1;
};

// Shared-memory layout of the FP32 kernels: X, S1 and S2 in three regions, each with its
// own per-element stride, so that the stride of each region can place the elements that
// share a warp on different banks without constraining the other two.  Line and plane
// strides and the pads come from an exhaustive search of a model of every warp access of
// variants 1 and 2 (gather store; stages 1, 2, 3, 2^T, 1^T; elements dealt over the
// block) at NE0 and NE0 / 2 elements per block, the shared memory per element held at or
// below the plain layout's (more costs variant 3 a block per SM at p = 4).  The model
// reproduces the shared-memory wavefront count that ncu reports for p = 4 (189 per
// element before, 168 after); measured on B300 the action gets 2-6 % faster for p <= 4.
struct SmemPick {
  int xl, xpad, q1, cs, s1pad, p2, s2pad;
};
constexpr SmemPick smem_pick(int P, int Q, bool DIFF) {
  return (P == 1 && Q == 2 && DIFF) ? SmemPick{2, 4, 3, 6, 4, 6, 0}
         : (P == 1 && Q == 2 && !DIFF) ? SmemPick{2, 4, 3, 6, 0, 6, 0}
         : (P == 1 && Q == 3 && DIFF) ? SmemPick{5, 0, 3, 14, 4, 29, 27}
         : (P == 1 && Q == 3 && !DIFF) ? SmemPick{2, 0, 3, 14, 0, 29, 15}
         : (P == 2 && Q == 3 && DIFF) ? SmemPick{3, 0, 5, 35, 0, 35, 0}
         : (P == 2 && Q == 3 && !DIFF) ? SmemPick{3, 0, 5, 35, 0, 35, 0}
         : (P == 2 && Q == 4 && DIFF) ? SmemPick{3, 0, 5, 20, 4, 20, 8}
         : (P == 2 && Q == 4 && !DIFF) ? SmemPick{3, 0, 5, 20, 0, 20, 0}
         : (P == 3 && Q == 4 && DIFF) ? SmemPick{5, 0, 5, 20, 16, 20, 0}
         : (P == 3 && Q == 4 && !DIFF) ? SmemPick{5, 0, 5, 20, 0, 20, 0}
         : (P == 3 && Q == 5 && DIFF) ? SmemPick{5, 0, 8, 37, 12, 26, 1}
         : (P == 3 && Q == 5 && !DIFF) ? SmemPick{5, 0, 8, 37, 0, 26, 17}
         : (P == 4 && Q == 5 && DIFF) ? SmemPick{5, 0, 7, 37, 7, 37, 14}
         : (P == 4 && Q == 5 && !DIFF) ? SmemPick{5, 0, 7, 37, 0, 37, 0}
         : (P == 4 && Q == 6 && DIFF) ? SmemPick{5, 0, 7, 38, 2, 38, 4}
         : (P == 4 && Q == 6 && !DIFF) ? SmemPick{5, 0, 9, 45, 0, 38, 0}
         // p = 6, 8 and mass p = 7 (q = p + 2): S1 strides from a search over the two S1 access
         // patterns alone (stage 1's lines (b, c) and stage 2's lines (i, c), one element): with the
         // plain strides stage 2's reads and 2^T's writes took up to 3.7x the wavefronts of a
         // conflict-free access (ncu at p = 8: 32 % of the shared wavefronts were bank conflicts);
         // these cut that to 1.5-1.7x for 18-67 % more S1.  Measured on B300 (best variant, ~3e7
         // DOFs): mass p = 6, 7, 8 -2.7, -2.2, -4.9 %, diffusion p = 6, 8 -3.0, -1.4 %; diffusion
         // p = 7 +4.6 % (kept plain), 1e5-DOF meshes within 2 %.
         // p = 5, q = 7: the plain strides with element pads for S1 and S2 from a model of stages
         // 1, 2, 3, 2^T, 1^T and the gather / scatter with the block's 5 (variant 1) or 2 (variant 2)
         // elements, whose 49-thread columns make every warp straddle two elements: the S2 pad moves
         // the second element's stage-3 columns onto the banks the first leaves free (modelled shared
         // wavefronts of a 5-element diffusion block 1,666 -> 1,414).  Measured on B300 (~3e7 DOFs,
         // two runs): diffusion -1.9 % (best plain), -2.4 % (the CG loop's fused build); mass -0.5..-1.1 %.
         : (P == 5 && Q == 7 && DIFF) ? SmemPick{7, 0, 7, 42, 3, 71, 19}
         : (P == 5 && Q == 7 && !DIFF) ? SmemPick{7, 0, 7, 42, 31, 71, 7}
         : (P == 6 && Q == 8) ? SmemPick{7, 0, 15, 105, 0, 72, 0}
         : (P == 7 && Q == 9 && !DIFF) ? SmemPick{9, 0, 12, 105, 0, 105, 0}
         : (P == 8 && Q == 10) ? SmemPick{9, 0, 13, 117, 0, 106, 0}
         // other p >= 5: the plain odd strides (the model-search picks of p <= 4's kind measured no
         // faster there, p = 8 diffusion 2-4 % slower)
         : SmemPick{(P + 1) | 1, 0, Q | 1, (P + 1) * (Q | 1), 0,
                    Q * Q + (((Q - (Q * Q) % 32) % 32) + 32) % 32, 0};
}

template <int P, int Q, bool DIFF>
struct F32Smem {
  static constexpr SmemPick K = smem_pick(P, Q, DIFF);
  static constexpr int N = P + 1;
  static constexpr int NC = DIFF ? 6 : 1;
  static constexpr int Q3 = Q * Q * Q;
  static constexpr int DSTRIDE = (Q3 + 3) & ~3;  // floats per stored D component (16-byte multiple)
  static constexpr int DELEM = NC * DSTRIDE;     // floats of D per element
  static constexpr int NC1 = DIFF ? 2 : 1;
  static constexpr int NC2 = DIFF ? 3 : 1;
  static constexpr int XL = K.xl;               // X [c][b][a]: line (b,c) at stride XL
  static constexpr int XE = XL * N * N + K.xpad;  // X region per element
  static constexpr int Q1 = K.q1;               // S1 [m][c][b][i]: entry (b,c,i) at b*Q1 + c*CS + i
  static constexpr int CS = K.cs;
  static constexpr int S1C = CS * N;            // one S1 component
  static constexpr int W1 = NC1 * S1C + K.s1pad;  // S1 region per element
  static constexpr int P2 = K.p2;               // S2 [m][c][j][i]: plane c at stride P2
  static constexpr int S2C = P2 * N;            // one S2 component
  static constexpr int W2 = NC2 * S2C + K.s2pad;  // S2 region per element
  static_assert(XL >= N && Q1 >= Q && CS >= N * Q1 && P2 >= Q * Q, "layout strides");
  static constexpr int TPE = Q * Q;
  static constexpr int NE0 = (256 / TPE) > 0 ? (256 / TPE) : 1;
};

// Launch shape of variants 0-2.
template <int P, int Q, bool DIFF, bool STAGE_D = true, int NE_DIV = 1>
struct TmaShape : F32Smem<P, Q, DIFF> {
  using L = F32Smem<P, Q, DIFF>;
  static constexpr int NE = (L::NE0 / NE_DIV) > 0 ? (L::NE0 / NE_DIV) : 1;
  static constexpr int SMEM = 16 + NE * ((STAGE_D ? L::DELEM : 0) + L::XE + L::W1 + L::W2) * 4;
};

// Launch shape of variant 3 (double-buffered D, x and map per block).
template <int P, int Q, bool DIFF>
struct PipeShape : F32Smem<P, Q, DIFF> {
  using L = F32Smem<P, Q, DIFF>;
  static constexpr int NE = L::NE0;
  static constexpr int T = L::TPE * NE;
  static constexpr int IDX = NE * L::N * L::N * L::N;  // map entries per group
  static constexpr int IDXR = (IDX + T - 1) / T;       // per thread
  static constexpr int SMEM = 16 + 2 * NE * L::DELEM * 4 + 2 * NE * L::XE * 4 + 2 * IDX * 4 + NE * (L::W1 + L::W2) * 4;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr int WAIT_LIMIT = 1 << 22;  // try_wait polls before a bounded wait gives up

// Poll limit of the first wait of a block for its staged D (fepa_test_set_first_wait_limit
// lowers it to make the timeout path run; the drain waits after a timeout keep WAIT_LIMIT).
__constant__ int c_first_wait_limit = WAIT_LIMIT;

// Bounded wait for the given phase parity of the barrier: false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity = 0, int limit = WAIT_LIMIT) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// asynchronous 4-byte global -> shared copy (no register round trip)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// one thread asks the TMA engine to pull [p, p + bytes) into L2 (p and bytes multiples of 16)
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch of [p, p + bytes) widened to 16-byte boundaries (every allocation of this
// library is 256-byte aligned and carries 16 bytes of slack past its end)
__device__ __forceinline__ void prefetch_range(const void* p, size_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t lo = a & ~(uintptr_t)15, hi = (a + bytes + 15) & ~(uintptr_t)15;
  bulk_prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
}

// L2 prefetch of an element group's D block (PF >= 1) and map entries (PF >= 2), issued
// by one thread when the block starts so the later loads hit L2
template <int PF>
__device__ __forceinline__ void prefetch_group(const void* d, size_t dbytes, const int* g, int nidx) {
  if (PF >= 1) prefetch_range(d, dbytes);
  if (PF >= 2) prefetch_range(g, 4u * (size_t)nidx);
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---------------------------------------------------------------------------
// stages (called by every thread of the block; `tid` is the work item's line within
// its element, `live` whether its element exists).  Stages 1, 2, 2^T and 1^T have
// fewer lines per element (n^2, Q n) than the element has threads (Q^2).  FLAT: the
// block deals their lines out over all its threads, so idle lanes gather in the last
// warps, which then skip the stage, instead of sitting in every warp.  Measured on
// B300 (with the L2 prefetch): p=2 8 %, p=4 2 % faster; p=6, 8 10-19 % slower
// (no warp is saved there and the straddled elements cost more), so p <= 4 only.
// ---------------------------------------------------------------------------

// work item of a stage with W lines per element: (element, line) of thread (tid, el)
template <bool FLAT, int W, int TPE>
__device__ __forceinline__ void stage_item(int tid, int el, int& e, int& line) {
  if (FLAT) {
    const int f = el * TPE + tid;
    e = f / W;
    line = f - e * W;
  } else {
    e = el;
    line = tid;  // lines >= W: the stage's own check leaves them idle
  }
}

// stage 1 (x): line (b,c) -> S1[m][c][b][i] for all i
template <int P, int Q, bool DIFF>
__device__ __forceinline__ void f32_stage1(int tid, bool live, const float* sX, float* S1) {
  using L = F32Smem<P, Q, DIFF>;
  using T = Tab32<P, Q>;
  constexpr int n = L::N;
  if (!(live && tid < n * n)) return;
  float xv[n];
#pragma unroll
  for (int a = 0; a < n; ++a) xv[a] = sX[tid * L::XL + a];
  float* o = S1 + (L::CS == n * L::Q1 ? tid * L::Q1 : (tid % n) * L::Q1 + (tid / n) * L::CS);
  if constexpr (!Pack32<P, Q, DIFF>::S1) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float sb = 0.f, sg = 0.f;
#pragma unroll
      for (int a = 0; a < n; ++a) {
        sb = fmaf(T::B(i, a), xv[a], sb);
        if (DIFF) sg = fmaf(T::G(i, a), xv[a], sg);
      }
      o[i] = sb;
      if (DIFF) o[L::S1C + i] = sg;
    }
    return;
  }
  // outputs i, i+1 in one packed FMA per input (each output's sum in the order of a)
#pragma unroll
  for (int ip = 0; ip < T::QH; ++ip) {
    float2 sb = make_float2(0.f, 0.f), sg = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < n; ++a) {
      sb = __ffma2_rn(T::Br(ip, a), bcast2(xv[a]), sb);
      if (DIFF) sg = __ffma2_rn(T::Gr(ip, a), bcast2(xv[a]), sg);
    }
    o[2 * ip] = sb.x;
    if (DIFF) o[L::S1C + 2 * ip] = sg.x;
    if (2 * ip + 1 < Q) {
      o[2 * ip + 1] = sb.y;
      if (DIFF) o[L::S1C + 2 * ip + 1] = sg.y;
    }
  }
}

// stage 2 (y): line (i,c) -> S2[m][c][j][i] for all j
//   DIFF: m=0 (x:G,y:B), m=1 (x:B,y:G), m=2 (x:B,y:B); mass: m=0 (B,B)
template <int P, int Q, bool DIFF>
__device__ __forceinline__ void f32_stage2(int tid, bool live, const float* S1, float* S2) {
  using L = F32Smem<P, Q, DIFF>;
  using T = Tab32<P, Q>;
  constexpr int n = L::N;
  if (!(live && tid < Q * n)) return;
  const int i = tid % Q, c = tid / Q;
  float vb[n], vg[n];
#pragma unroll
  for (int b = 0; b < n; ++b) {
    vb[b] = S1[b * L::Q1 + c * L::CS + i];
    if (DIFF) vg[b] = S1[L::S1C + b * L::Q1 + c * L::CS + i];
  }
  if constexpr (!Pack32<P, Q, DIFF>::S2) {
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      float bb = 0.f, bg = 0.f, gb = 0.f;
#pragma unroll
      for (int b = 0; b < n; ++b) {
        bb = fmaf(T::B(j, b), vb[b], bb);
        if (DIFF) {
          bg = fmaf(T::G(j, b), vb[b], bg);
          gb = fmaf(T::B(j, b), vg[b], gb);
        }
      }
      const int o = c * L::P2 + j * Q + i;
      if (DIFF) {
        S2[o] = gb;
        S2[L::S2C + o] = bg;
        S2[2 * L::S2C + o] = bb;
      } else {
        S2[o] = bb;
      }
    }
    return;
  }
#pragma unroll
  for (int jp = 0; jp < T::QH; ++jp) {
    float2 bb = make_float2(0.f, 0.f), bg = bb, gb = bb;
#pragma unroll
    for (int b = 0; b < n; ++b) {
      bb = __ffma2_rn(T::Br(jp, b), bcast2(vb[b]), bb);
      if (DIFF) {
        bg = __ffma2_rn(T::Gr(jp, b), bcast2(vb[b]), bg);
        gb = __ffma2_rn(T::Br(jp, b), bcast2(vg[b]), gb);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * jp + h;
      if (j >= Q) break;
      const int o = c * L::P2 + j * Q + i;
      if (DIFF) {
        S2[o] = h ? gb.y : gb.x;
        S2[L::S2C + o] = h ? bg.y : bg.x;
        S2[2 * L::S2C + o] = h ? bb.y : bb.x;
      } else {
        S2[o] = h ? bb.y : bb.x;
      }
    }
  }
}

// stage 3 (z) + D + stage 3^T, one (i,j) column per thread, in registers, in scalar FMAs
// (one point at a time); D at dE (shared or global), component stride DSTRIDE, point k at
// dE[k*Q*Q].  PRE: the column's D was loaded into dpre[k * NCD + m] before the preceding barrier
template <int P, int Q, bool DIFF, bool PRE = false>
__device__ __forceinline__ void f32_stage3_scalar(int tid, bool live, float* S2, const float* dE, const float* dpre = nullptr) {
  using L = F32Smem<P, Q, DIFF>;
  using T = Tab32<P, Q>;
  constexpr int n = L::N;
  if (!live) return;
  float c0[n], c1[n], c2[n], a0[n], a1[n], a2[n];
#pragma unroll
  for (int c = 0; c < n; ++c) {
    c0[c] = S2[c * L::P2 + tid];
    if (DIFF) {
      c1[c] = S2[L::S2C + c * L::P2 + tid];
      c2[c] = S2[2 * L::S2C + c * L::P2 + tid];
    }
    a0[c] = 0.f;
    if (DIFF) a1[c] = a2[c] = 0.f;
  }
  // D of point k+1 is loaded while point k is computed (one step of software pipelining)
  constexpr int NCD = DIFF ? 6 : 1;
  float dn[NCD];
  if (!PRE) {
#pragma unroll
    for (int m = 0; m < NCD; ++m) dn[m] = dE[m * L::DSTRIDE];
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    float dc[NCD];
    if (PRE) {
#pragma unroll
      for (int m = 0; m < NCD; ++m) dc[m] = dpre[k * NCD + m];
    } else {
#pragma unroll
      for (int m = 0; m < NCD; ++m) dc[m] = dn[m];
      if (k + 1 < Q) {
#pragma unroll
        for (int m = 0; m < NCD; ++m) dn[m] = dE[(k + 1) * Q * Q + m * L::DSTRIDE];
      }
    }
    if (DIFF) {
      float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
      for (int c = 0; c < n; ++c) {
        u0 = fmaf(T::B(k, c), c0[c], u0);
        u1 = fmaf(T::B(k, c), c1[c], u1);
        u2 = fmaf(T::G(k, c), c2[c], u2);
      }
      const float d00 = dc[0], d01 = dc[1 % NCD], d02 = dc[2 % NCD], d11 = dc[3 % NCD], d12 = dc[4 % NCD],
                  d22 = dc[5 % NCD];
      const float v0 = fmaf(d00, u0, fmaf(d01, u1, d02 * u2));
      const float v1 = fmaf(d01, u0, fmaf(d11, u1, d12 * u2));
      const float v2 = fmaf(d02, u0, fmaf(d12, u1, d22 * u2));
#pragma unroll
      for (int c = 0; c < n; ++c) {
        a0[c] = fmaf(T::B(k, c), v0, a0[c]);
        a1[c] = fmaf(T::B(k, c), v1, a1[c]);
        a2[c] = fmaf(T::G(k, c), v2, a2[c]);
      }
    } else {
      float u = 0.f;
#pragma unroll
      for (int c = 0; c < n; ++c) u = fmaf(T::B(k, c), c0[c], u);
      const float v = dc[0] * u;
#pragma unroll
      for (int c = 0; c < n; ++c) a0[c] = fmaf(T::B(k, c), v, a0[c]);
    }
  }
  // each thread overwrites only its own column
#pragma unroll
  for (int c = 0; c < n; ++c) {
    S2[c * L::P2 + tid] = a0[c];
    if (DIFF) {
      S2[L::S2C + c * L::P2 + tid] = a1[c];
      S2[2 * L::S2C + c * L::P2 + tid] = a2[c];
    }
  }
}

// stage 3 (z) + D + stage 3^T, one (i,j) column per thread, in registers, by the policy of
// Pack32: points paired in packed FMAs, or only the transposed contraction's columns paired
// (bits 2, 3), else the scalar form above; arguments as there
template <int P, int Q, bool DIFF, bool PRE = false>
__device__ __forceinline__ void f32_stage3(int tid, bool live, float* S2, const float* dE, const float* dpre = nullptr) {
  using L = F32Smem<P, Q, DIFF>;
  using T = Tab32<P, Q>;
  constexpr int n = L::N;
  if constexpr (!Pack32<P, Q, DIFF>::S3T) {
    f32_stage3_scalar<P, Q, DIFF, PRE>(tid, live, S2, dE, dpre);
    return;
  }
  if (!live) return;
  float c0[n], c1[n], c2[n];
#pragma unroll
  for (int c = 0; c < n; ++c) {
    c0[c] = S2[c * L::P2 + tid];
    if (DIFF) {
      c1[c] = S2[L::S2C + c * L::P2 + tid];
      c2[c] = S2[2 * L::S2C + c * L::P2 + tid];
    }
  }
  // transposed-stage accumulators: columns (2cp, 2cp+1) as pairs, column n-1 alone when n is odd
  constexpr int NP = n / 2;
  constexpr bool ODDN = (n & 1) != 0;
  float2 A0[NP], A1[NP], A2[NP];
  float z0 = 0.f, z1 = 0.f, z2 = 0.f;
#pragma unroll
  for (int cp = 0; cp < NP; ++cp) {
    A0[cp] = make_float2(0.f, 0.f);
    if (DIFF) A1[cp] = A2[cp] = A0[cp];
  }
  // D of point k+1 is loaded while point k is computed (one step of software pipelining)
  constexpr int NCD = DIFF ? 6 : 1;
  float dn[NCD];
  if (!PRE) {
#pragma unroll
    for (int m = 0; m < NCD; ++m) dn[m] = dE[m * L::DSTRIDE];
  }
  constexpr bool PF = Pack32<P, Q, DIFF>::S3F, PT = Pack32<P, Q, DIFF>::S3T;
#pragma unroll
  for (int kp = 0; kp < T::QH; ++kp) {
    // points 2kp, 2kp+1 of the column in packed FMAs
    float2 U0 = make_float2(0.f, 0.f), U1 = U0, U2 = U0;
    if (PF) {
#pragma unroll
    for (int c = 0; c < n; ++c) {
      U0 = __ffma2_rn(T::Br(kp, c), bcast2(c0[c]), U0);
      if (DIFF) {
        U1 = __ffma2_rn(T::Br(kp, c), bcast2(c1[c]), U1);
        U2 = __ffma2_rn(T::Gr(kp, c), bcast2(c2[c]), U2);
      }
    }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * kp + h;
      if (k >= Q) break;
      if (!PF) {
        float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
        for (int c = 0; c < n; ++c) {
          u0 = fmaf(T::B(k, c), c0[c], u0);
          if (DIFF) {
            u1 = fmaf(T::B(k, c), c1[c], u1);
            u2 = fmaf(T::G(k, c), c2[c], u2);
          }
        }
        if (h) { U0.y = u0; U1.y = u1; U2.y = u2; } else { U0.x = u0; U1.x = u1; U2.x = u2; }
      }
      float dc[NCD];
      if (PRE) {
#pragma unroll
        for (int m = 0; m < NCD; ++m) dc[m] = dpre[k * NCD + m];
      } else {
#pragma unroll
        for (int m = 0; m < NCD; ++m) dc[m] = dn[m];
        if (k + 1 < Q) {
#pragma unroll
          for (int m = 0; m < NCD; ++m) dn[m] = dE[(k + 1) * Q * Q + m * L::DSTRIDE];
        }
      }
      if (DIFF) {
        const float u0 = h ? U0.y : U0.x, u1 = h ? U1.y : U1.x, u2 = h ? U2.y : U2.x;
        const float d00 = dc[0], d01 = dc[1 % NCD], d02 = dc[2 % NCD], d11 = dc[3 % NCD], d12 = dc[4 % NCD],
                    d22 = dc[5 % NCD];
        const float v0 = fmaf(d00, u0, fmaf(d01, u1, d02 * u2));
        const float v1 = fmaf(d01, u0, fmaf(d11, u1, d12 * u2));
        const float v2 = fmaf(d02, u0, fmaf(d12, u1, d22 * u2));
#pragma unroll
        for (int cp = 0; cp < NP; ++cp) {
          if (PT) {
            A0[cp] = __ffma2_rn(T::Bc(k, cp), bcast2(v0), A0[cp]);
            A1[cp] = __ffma2_rn(T::Bc(k, cp), bcast2(v1), A1[cp]);
            A2[cp] = __ffma2_rn(T::Gc(k, cp), bcast2(v2), A2[cp]);
          } else {
            A0[cp].x = fmaf(T::Bc(k, cp).x, v0, A0[cp].x);
            A0[cp].y = fmaf(T::Bc(k, cp).y, v0, A0[cp].y);
            A1[cp].x = fmaf(T::Bc(k, cp).x, v1, A1[cp].x);
            A1[cp].y = fmaf(T::Bc(k, cp).y, v1, A1[cp].y);
            A2[cp].x = fmaf(T::Gc(k, cp).x, v2, A2[cp].x);
            A2[cp].y = fmaf(T::Gc(k, cp).y, v2, A2[cp].y);
          }
        }
        if (ODDN) {
          z0 = fmaf(T::Bc(k, NP).x, v0, z0);
          z1 = fmaf(T::Bc(k, NP).x, v1, z1);
          z2 = fmaf(T::Gc(k, NP).x, v2, z2);
        }
      } else {
        const float v = dc[0] * (h ? U0.y : U0.x);
#pragma unroll
        for (int cp = 0; cp < NP; ++cp) {
          if (PT) {
            A0[cp] = __ffma2_rn(T::Bc(k, cp), bcast2(v), A0[cp]);
          } else {
            A0[cp].x = fmaf(T::Bc(k, cp).x, v, A0[cp].x);
            A0[cp].y = fmaf(T::Bc(k, cp).y, v, A0[cp].y);
          }
        }
        if (ODDN) z0 = fmaf(T::Bc(k, NP).x, v, z0);
      }
    }
  }
  // each thread overwrites only its own column
#pragma unroll
  for (int c = 0; c < n; ++c) {
    const bool last = ODDN && c == n - 1;
    const int cp = last ? 0 : c / 2;
    S2[c * L::P2 + tid] = last ? z0 : ((c & 1) ? A0[cp].y : A0[cp].x);
    if (DIFF) {
      S2[L::S2C + c * L::P2 + tid] = last ? z1 : ((c & 1) ? A1[cp].y : A1[cp].x);
      S2[2 * L::S2C + c * L::P2 + tid] = last ? z2 : ((c & 1) ? A2[cp].y : A2[cp].x);
    }
  }
}

// stage 2^T (y): line (i,c) -> S1[0][c][b][i] = sum_j B[j][b] A0,
//                             S1[1][c][b][i] = sum_j G[j][b] A1 + B[j][b] A2
template <int P, int Q, bool DIFF>
__device__ __forceinline__ void f32_stage2t(int tid, bool live, const float* S2, float* S1) {
  using L = F32Smem<P, Q, DIFF>;
  using T = Tab32<P, Q>;
  constexpr int n = L::N;
  if (!(live && tid < Q * n)) return;
  const int i = tid % Q, c = tid / Q;
  float v0[Q], v1[Q], v2[Q];
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    v0[j] = S2[c * L::P2 + j * Q + i];
    if (DIFF) {
      v1[j] = S2[L::S2C + c * L::P2 + j * Q + i];
      v2[j] = S2[2 * L::S2C + c * L::P2 + j * Q + i];
    }
  }
  if constexpr (!Pack32<P, Q, DIFF>::S2T) {
#pragma unroll
    for (int b = 0; b < n; ++b) {
      float t0 = 0.f, t1 = 0.f;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        t0 = fmaf(T::B(j, b), v0[j], t0);
        if (DIFF) t1 = fmaf(T::G(j, b), v1[j], fmaf(T::B(j, b), v2[j], t1));
      }
      S1[b * L::Q1 + c * L::CS + i] = t0;
      if (DIFF) S1[L::S1C + b * L::Q1 + c * L::CS + i] = t1;
    }
    return;
  }
  // outputs b, b+1 in one packed FMA per input (each output's sum in the order of j)
#pragma unroll
  for (int bp = 0; bp < T::NH; ++bp) {
    float2 t0 = make_float2(0.f, 0.f), t1 = t0;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      t0 = __ffma2_rn(T::Bc(j, bp), bcast2(v0[j]), t0);
      if (DIFF) t1 = __ffma2_rn(T::Gc(j, bp), bcast2(v1[j]), __ffma2_rn(T::Bc(j, bp), bcast2(v2[j]), t1));
    }
    S1[2 * bp * L::Q1 + c * L::CS + i] = t0.x;
    if (DIFF) S1[L::S1C + 2 * bp * L::Q1 + c * L::CS + i] = t1.x;
    if (2 * bp + 1 < n) {
      S1[(2 * bp + 1) * L::Q1 + c * L::CS + i] = t0.y;
      if (DIFF) S1[L::S1C + (2 * bp + 1) * L::Q1 + c * L::CS + i] = t1.y;
    }
  }
}

// stage 1^T arithmetic of one line: s[a] = sum_i G[i][a] t0[i] + B[i][a] t1[i] (diffusion) or
// sum_i B[i][a] t0[i] (mass), outputs a, a+1 in one packed FMA per input
template <int P, int Q, bool DIFF>
__device__ __forceinline__ void f32_line1t(const float (&t0)[Q], const float (&t1)[Q], float (&s)[P + 1]) {
  using T = Tab32<P, Q>;
  constexpr int n = P + 1;
  if constexpr (!Pack32<P, Q, DIFF>::S1T) {
#pragma unroll
    for (int a = 0; a < n; ++a) {
      float v = 0.f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (DIFF)
          v = fmaf(T::G(i, a), t0[i], fmaf(T::B(i, a), t1[i], v));
        else
          v = fmaf(T::B(i, a), t0[i], v);
      }
      s[a] = v;
    }
    return;
  }
#pragma unroll
  for (int ap = 0; ap < T::NH; ++ap) {
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (DIFF)
        v = __ffma2_rn(T::Gc(i, ap), bcast2(t0[i]), __ffma2_rn(T::Bc(i, ap), bcast2(t1[i]), v));
      else
        v = __ffma2_rn(T::Bc(i, ap), bcast2(t0[i]), v);
    }
    s[2 * ap] = v.x;
    if (2 * ap + 1 < n) s[2 * ap + 1] = v.y;
  }
}

// stage 1^T (x) and G^T: line (b,c) -> y[g(a,b,c)] += sum_i G[i][a] T0 + B[i][a] T1.
// gl: the element's n^3 map entries (global or shared memory).
template <int P, int Q, bool DIFF>
__device__ __forceinline__ void f32_stage1t(int tid, bool live, const float* S1, const int* gl,
                                            const float* __restrict__ x, float* __restrict__ y) {
  using L = F32Smem<P, Q, DIFF>;
  using T = Tab32<P, Q>;
  constexpr int n = L::N;
  if (!(live && tid < n * n)) return;
  float t0[Q], t1[Q];
  const float* in = S1 + (L::CS == n * L::Q1 ? tid * L::Q1 : (tid % n) * L::Q1 + (tid / n) * L::CS);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    t0[i] = in[i];
    if (DIFF) t1[i] = in[L::S1C + i];
  }
  float sv[n];
  f32_line1t<P, Q, DIFF>(t0, t1, sv);
#pragma unroll
  for (int a = 0; a < n; ++a) {
    const float s = sv[a];
    const int gi = gl[a + n * tid];
    if (gi >= 0) {
      atomicAdd(y + gi, s);
    } else if (!((~gi) & ESS_SKIP)) {
      atomicAdd(y + (~gi), x[~gi]);
    }
  }
}

// stage 1^T (x) and G^T into shared memory: line (b,c) -> Y[c][b][a] (X's layout) for
// the scatter that follows in element-local DOF order (coalesced map loads and atomics)
// DOT: before a result overwrites the gathered input at the same place, the product of
// the two is added to acc: the line's share of (x, A x).  (A plain FP32 sum of n terms:
// its rounding is of the order of that already in the FP32 results themselves.)  Formed
// here rather than as u^T D u at the points of stage 3: that build, measured on B300 at
// BP3 p = 4, was 14 % slower (its register allocation changed), this one 5 %.
template <int P, int Q, bool DIFF, bool DOT = false>
__device__ __forceinline__ void f32_stage1t_smem(int tid, bool live, const float* S1, float* Y, float& acc) {
  using L = F32Smem<P, Q, DIFF>;
  using T = Tab32<P, Q>;
  constexpr int n = L::N;
  if (!(live && tid < n * n)) return;
  float t0[Q], t1[Q];
  const float* in = S1 + (L::CS == n * L::Q1 ? tid * L::Q1 : (tid % n) * L::Q1 + (tid / n) * L::CS);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    t0[i] = in[i];
    if (DIFF) t1[i] = in[L::S1C + i];
  }
  float sv[n];
  f32_line1t<P, Q, DIFF>(t0, t1, sv);
#pragma unroll
  for (int a = 0; a < n; ++a) {
    if (DOT) acc = fmaf(Y[tid * L::XL + a], sv[a], acc);
    Y[tid * L::XL + a] = sv[a];
  }
}

// DOT: each warp sums its threads' shares (the block's last warp may be partial: lanes
// past the block's end do not exist and are left out) and lane 0 adds the warp's sum by
// one double atomic to a slot (the CG update kernel sums the DOT_SLOTS slots)
constexpr int DOT_SLOTS = RED_THREADS;
__device__ __forceinline__ void dot_publish(float acc, int nthreads, int flat, double* dot) {
  const int lane = flat & 31, w = flat >> 5;
  const int nl = min(32, nthreads - 32 * w);
  const unsigned mask = nl == 32 ? 0xffffffffu : ((1u << nl) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float t = __shfl_down_sync(mask, acc, o);
    if (lane + o < nl) acc += t;
  }
  if (lane == 0) atomicAdd(dot + (blockIdx.x * ((nthreads + 31) / 32) + w) % DOT_SLOTS, (double)acc);
}

// ---------------------------------------------------------------------------
// variants 0-2: one element group per block
// ---------------------------------------------------------------------------
// PF: L2 prefetch at block start (TMA engine, one thread): 1 = the group's D (unless staged),
// 2 = also its map entries.  Measured on B300: 4-11 % faster for p = 2..8 (PF 2 best).
// DEARLY (measured): loading the stage-3 D column before the barrier is 3-6 % faster for
// p <= 3 and 3-17 % slower from p = 4 (the 6 q registers it holds cost occupancy there).
// BSKIP: the batched build, which reads elem_prob / prob_done (a separate instantiation, so
// the single-operator kernels carry none of its checks: they cost those 5 % when tested).
// The block's work on one tile of ne <= NE consecutive elements starting at e0 (called once per
// block by pa_apply_f32_tma, or per tile of a work list by pa_apply_f32_tiles)
template <int P, int Q, bool DIFF, bool STAGE_D, int NE_DIV, int PF = 2, bool FLAT = (P <= 4), bool DEARLY = (P <= 3),
          bool BSKIP = false, bool DOT = false>
__device__ __forceinline__ void f32_tile(int64_t e0, int ne, const int* __restrict__ gmap,
                                         const float* __restrict__ qd32, const float* __restrict__ x,
                                         float* __restrict__ y, const int* __restrict__ elem_prob,
                                         const int* __restrict__ prob_done, int* __restrict__ err,
                                         double* __restrict__ dot) {
  using S = TmaShape<P, Q, DIFF, STAGE_D, NE_DIV>;
  constexpr int n = S::N, TPE = S::TPE, NE = S::NE;
  static_assert(!DOT || (P >= 3 && !BSKIP), "the fused (x, A x) needs the shared-memory scatter");
  extern __shared__ __align__(16) unsigned char smem_tma[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_tma);
  float* sD = reinterpret_cast<float*>(smem_tma + 16);
  float* sXall = sD + (STAGE_D ? NE * S::DELEM : 0);  // [NE][XE]
  float* sS1 = sXall + NE * S::XE;                     // [NE][W1]
  float* sS2 = sS1 + NE * S::W1;                       // [NE][W2]
  const int tid = threadIdx.x, el = threadIdx.y;
  // batched problems (BSKIP): the elements of a converged problem do no work, and a block
  // whose elements all belong to converged problems leaves at once
  auto alive = [&](int e) { return e < ne && !(BSKIP && prob_done[elem_prob[e0 + e]]); };
  if (BSKIP && !__syncthreads_or(alive(el))) return;
  if (PF > 0 && tid == 0 && el == 0) {
    if (!STAGE_D) prefetch_range(qd32 + e0 * S::DELEM, (size_t)ne * S::DELEM * 4u);
    if (PF >= 2) prefetch_range(gmap + e0 * (n * n * n), 4u * (size_t)ne * n * n * n);
  }
  if (STAGE_D && tid == 0 && el == 0) {
    mbar_init(mbar, 1);
    const uint32_t bytes = (uint32_t)ne * S::DELEM * 4u;
    mbar_expect_tx(mbar, bytes);
    bulk_copy_g2s(sD, qd32 + e0 * S::DELEM, bytes, mbar);
  }
  // FLATG (p = 3, 4): the gather and the local-order scatter run over the block's element-local
  // DOFs as one flat range (the group's map entries are contiguous), so no warp's map loads
  // straddle two elements.  Measured on B300: p = 3, 4 1-2 % faster; p = 2 2-7 %, p = 6 7 %,
  // p = 8 up to 38 % slower (elsewhere the per-element form is kept).
  constexpr bool FLATG = (P == 3 || P == 4);
  constexpr int N3 = n * n * n, TB = TPE * NE, GR = (N3 * NE + TB - 1) / TB;
  const int flat = el * TPE + tid;
  const int* gblk = gmap + e0 * N3;
  const bool live = alive(el);
  float* sX = sXall + el * S::XE;
  const int* g = gmap + (e0 + el) * N3;
  if constexpr (FLATG) {
    int gi[GR];
    float xv[GR];
#pragma unroll
    for (int r = 0; r < GR; ++r) {
      const int f = flat + r * TB;
      gi[r] = (f < ne * N3 && (!BSKIP || alive(f / N3))) ? __ldg(gblk + f) : -1;
    }
#pragma unroll
    for (int r = 0; r < GR; ++r) xv[r] = gi[r] >= 0 ? __ldg(x + gi[r]) : 0.f;
#pragma unroll
    for (int r = 0; r < GR; ++r) {
      const int f = flat + r * TB;
      if (f < ne * N3) {
        const int e = f / N3, l = f - e * N3;
        sXall[e * S::XE + (l / n) * S::XL + l % n] = xv[r];
      }
    }
  } else if (live) {
    // gather: all map loads first, then all x loads, so the dependent pairs overlap
    constexpr int GRE = (N3 + TPE - 1) / TPE;
    int gi[GRE];
    float xv[GRE];
#pragma unroll
    for (int r = 0; r < GRE; ++r) {
      const int l = tid + r * TPE;
      gi[r] = l < N3 ? __ldg(g + l) : -1;
    }
#pragma unroll
    for (int r = 0; r < GRE; ++r) xv[r] = gi[r] >= 0 ? __ldg(x + gi[r]) : 0.f;
#pragma unroll
    for (int r = 0; r < GRE; ++r) {
      const int l = tid + r * TPE;
      if (l < N3) sX[(l / n) * S::XL + l % n] = xv[r];
    }
  }
  __syncthreads();
  {
    int e, ln;
    stage_item<FLAT, n * n, TPE>(tid, el, e, ln);
    f32_stage1<P, Q, DIFF>(ln, alive(e), sXall + e * S::XE, sS1 + e * S::W1);
  }
  __syncthreads();
  {
    int e, ln;
    stage_item<FLAT, Q * n, TPE>(tid, el, e, ln);
    f32_stage2<P, Q, DIFF>(ln, alive(e), sS1 + e * S::W1, sS2 + e * S::W2);
  }
  // DEARLY: the stage-3 thread loads its whole D column before the barrier, so the loads
  // overlap the wait for the other threads' stage 2
  constexpr int NCD = DIFF ? 6 : 1;
  float dpre[(DEARLY && !STAGE_D) ? NCD * Q : 1];
  if (DEARLY && !STAGE_D && alive(el)) {
    const float* dg = qd32 + (e0 + el) * S::DELEM + tid;
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
      for (int m = 0; m < NCD; ++m) dpre[k * NCD + m] = __ldg(dg + k * Q * Q + m * S::DSTRIDE);
  }
  if (STAGE_D) {
    // D must have landed before stage 3; every thread observes the barrier (bounded)
    const bool ok = mbar_wait_bounded(mbar, 0, c_first_wait_limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && el == 0) {
        atomicOr(err, 1);
        mbar_wait_bounded(mbar);  // let the copy in flight finish before the block exits
      }
      return;
    }
  } else {
    __syncthreads();
  }
  // stage-3 columns: when an element's Q^2 columns are not a whole number of warps, the
  // first NE * 32W threads can take columns 0..32W-1 element by element (whole warps on one
  // element: contiguous S2 and D) and the rest the tails, so that only one warp spans
  // elements (modelled: 17 % fewer stage-3 shared wavefronts at p = 4).  Measured on B300:
  // 2.8 % faster at Q = 6 (BP3 p = 4), 3.3 % at Q = 10, neutral at Q = 7, 3 % slower at
  // Q = 9 -- used for Q = 6 and 10.
  int e3 = el, c3 = tid;
  if constexpr ((Q == 6 || Q == 10) && !DEARLY) {
    constexpr int W = TPE / 32, TT = TPE - 32 * W;
    const int flat = el * TPE + tid;
    if (flat < NE * 32 * W) {
      e3 = flat / (32 * W);
      c3 = flat - e3 * (32 * W);
    } else {
      const int f = flat - NE * 32 * W;
      e3 = f / TT;
      c3 = 32 * W + (f - e3 * TT);
    }
  }
  const float* dE = (STAGE_D ? sD + e3 * S::DELEM : qd32 + (e0 + e3) * S::DELEM) + c3;
  f32_stage3<P, Q, DIFF, DEARLY && !STAGE_D>(c3, alive(e3), sS2 + e3 * S::W2, dE, dpre);
  __syncthreads();
  {
    int e, ln;
    stage_item<FLAT, Q * n, TPE>(tid, el, e, ln);
    f32_stage2t<P, Q, DIFF>(ln, alive(e), sS2 + e * S::W2, sS1 + e * S::W1);
  }
  __syncthreads();
  // YSM: stage 1^T writes the element results into the (free) X buffer and the block then
  // scatters them in element-local DOF order like the gather, so the map loads and the
  // atomics are coalesced over consecutive DOFs instead of strided by lines.  Measured on
  // B300: p = 3..8 2-14 % faster (mass p = 8 22 %), p = 1, 2 4-7 % slower.
  constexpr bool YSM = P >= 3;
  if (!YSM) {
    int e, ln;
    stage_item<FLAT, n * n, TPE>(tid, el, e, ln);
    f32_stage1t<P, Q, DIFF>(ln, alive(e), sS1 + e * S::W1, gmap + (e0 + e) * (n * n * n), x, y);
    return;
  }
  // DOT (the CG loop's build): (x, A x) = sum over elements of x_e . (A_e x_e) with x_e zero
  // at essential DOFs, plus x_g^2 for each essential DOF (the identity rows), so the
  // CG's separate (d, h) pass over two N-vectors is not needed
  float acc = 0.f;
  {
    int e, ln;
    stage_item<FLAT, n * n, TPE>(tid, el, e, ln);
    f32_stage1t_smem<P, Q, DIFF, DOT>(ln, alive(e), sS1 + e * S::W1, sXall + e * S::XE, acc);
  }
  __syncthreads();
  // scatter in element-local DOF order (over the block's flat range with FLATG), as the
  // gather: map loads first, then the atomics
  if constexpr (!FLATG) {
    if (live) {
      constexpr int GRE = (N3 + TPE - 1) / TPE;
      int gi[GRE];
#pragma unroll
      for (int r = 0; r < GRE; ++r) {
        const int l = tid + r * TPE;
        gi[r] = l < N3 ? __ldg(g + l) : 0;
      }
#pragma unroll
      for (int r = 0; r < GRE; ++r) {
        const int l = tid + r * TPE;
        if (l < N3) {
          const int gv = gi[r];
          if (gv >= 0) {
            atomicAdd(y + gv, sX[(l / n) * S::XL + l % n]);
          } else if (!((~gv) & ESS_SKIP)) {
            const float xe = x[~gv];
            atomicAdd(y + (~gv), xe);
            if (DOT) acc = fmaf(xe, xe, acc);
          }
        }
      }
    }
  } else {
    int gi[GR];
#pragma unroll
    for (int r = 0; r < GR; ++r) {
      const int f = flat + r * TB;
      gi[r] = f < ne * N3 ? __ldg(gblk + f) : 0;
    }
#pragma unroll
    for (int r = 0; r < GR; ++r) {
      const int f = flat + r * TB;
      const int e = f / N3, l = f - e * N3;
      if (f >= ne * N3 || (BSKIP && !alive(e))) continue;
      const int gv = gi[r];
      if (gv >= 0) {
        atomicAdd(y + gv, sXall[e * S::XE + (l / n) * S::XL + l % n]);
      } else if (!((~gv) & ESS_SKIP)) {
        const float xe = x[~gv];
        atomicAdd(y + (~gv), xe);
        if (DOT) acc = fmaf(xe, xe, acc);
      }
    }
  }
  if constexpr (DOT) dot_publish(acc, TPE * NE, el * TPE + tid, dot);
}

template <int P, int Q, bool DIFF, bool STAGE_D, int NE_DIV, int PF = 2, bool FLAT = (P <= 4), bool DEARLY = (P <= 3),
          bool BSKIP = false, bool DOT = false>
__global__ void __launch_bounds__(TmaShape<P, Q, DIFF, STAGE_D, NE_DIV>::TPE * TmaShape<P, Q, DIFF, STAGE_D, NE_DIV>::NE)
pa_apply_f32_tma(int E, const int* __restrict__ gmap, const float* __restrict__ qd32, const float* __restrict__ x,
                 float* __restrict__ y, const int* __restrict__ skip, const int* __restrict__ elem_prob,
                 const int* __restrict__ prob_done, int* __restrict__ err, double* __restrict__ dot) {
  constexpr int NE = TmaShape<P, Q, DIFF, STAGE_D, NE_DIV>::NE;
  if (skip && *skip) return;
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  f32_tile<P, Q, DIFF, STAGE_D, NE_DIV, PF, FLAT, DEARLY, BSKIP, DOT>(e0, (int)((E - e0) < NE ? (E - e0) : NE), gmap,
                                                                     qd32, x, y, elem_prob, prob_done, err, dot);
}

// Persistent form over a work list (the batch's iteration loop): a fixed grid walks the tiles
// act[0 .. *nact) of the table tiles (element offset, count <= NE) -- the tiles of problems still
// running -- so finished problems launch no blocks.  Direct D, in the shape of variant 1
// (NE_DIV 1) or 2 (NE_DIV 2), chosen per batch group by timing.
template <int P, int Q, bool DIFF, int NE_DIV>
__global__ void __launch_bounds__(TmaShape<P, Q, DIFF, false, NE_DIV>::TPE * TmaShape<P, Q, DIFF, false, NE_DIV>::NE)
pa_apply_f32_tiles(const int2* __restrict__ tiles, const int* __restrict__ act, const int* __restrict__ nact,
                   const int* __restrict__ gmap, const float* __restrict__ qd32, const float* __restrict__ x,
                   float* __restrict__ y, const int* __restrict__ skip, int* __restrict__ err) {
  if (skip && *skip) return;
  const int count = *nact;
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const int2 tl = tiles[act[i]];
    f32_tile<P, Q, DIFF, false, NE_DIV>(tl.x, tl.y, gmap, qd32, x, y, nullptr, nullptr, err, nullptr);
    __syncthreads();  // (the next tile reuses the shared buffers)
  }
}

// ---------------------------------------------------------------------------
// variant 3: persistent, software-pipelined over element groups (elem_prob and
// prob_done are not read: the batched solve does not select this variant)
// ---------------------------------------------------------------------------
template <int P, int Q, bool DIFF, bool FLAT = (P <= 4)>
__global__ void __launch_bounds__(PipeShape<P, Q, DIFF>::T)
pa_apply_f32_pipe(int E, const int* __restrict__ gmap, const float* __restrict__ qd32, const float* __restrict__ x,
                  float* __restrict__ y, const int* __restrict__ skip, const int* __restrict__ elem_prob,
                  const int* __restrict__ prob_done, int* __restrict__ err,
                  double* __restrict__ /*dot: not built here*/) {
  using S = PipeShape<P, Q, DIFF>;
  constexpr int n = S::N, n3 = n * n * n, TPE = S::TPE, NE = S::NE, T = S::T;
  if (skip && *skip) return;
  const int G = (E + NE - 1) / NE;
  int g = blockIdx.x;
  if (g >= G) return;
  extern __shared__ __align__(16) unsigned char smem_pipe[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_pipe);  // [2]
  float* sD = reinterpret_cast<float*>(smem_pipe + 16);     // [2][NE*DELEM]
  float* sX = sD + 2 * NE * S::DELEM;                       // [2][NE][XE]
  int* sI = reinterpret_cast<int*>(sX + 2 * NE * S::XE);    // [2][IDX]
  float* sS1 = reinterpret_cast<float*>(sI + 2 * S::IDX);   // [NE][W1]
  float* sS2 = sS1 + NE * S::W1;                            // [NE][W2]
  const int tid = threadIdx.x, el = threadIdx.y, flat = el * TPE + tid;
  float* S2 = sS2 + el * S::W2;

  // D of group gg into buffer b (one thread)
  auto issue_d = [&](int gg, int b) {
    const int64_t e0 = (int64_t)gg * NE;
    const int ne = (int)((E - e0) < NE ? (E - e0) : NE);
    const uint32_t bytes = (uint32_t)ne * S::DELEM * 4u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&mbar[b], bytes);
    bulk_copy_g2s(sD + b * NE * S::DELEM, qd32 + e0 * S::DELEM, bytes, &mbar[b]);
  };
  // map entries of group gg held by this thread
  auto load_idx = [&](int gg, int (&r)[S::IDXR]) {
    const int64_t base = (int64_t)gg * S::IDX;
    const int64_t lim = (int64_t)E * n3 - base;
#pragma unroll
    for (int k = 0; k < S::IDXR; ++k) {
      const int f = flat + k * T;
      r[k] = (f < S::IDX && f < lim) ? gmap[base + f] : 0;
    }
  };
  // store the map entries and gather x of group gg into buffer b (asynchronously)
  auto gather = [&](int gg, int b, const int (&r)[S::IDXR]) {
    const int64_t lim = (int64_t)E * n3 - (int64_t)gg * S::IDX;
#pragma unroll
    for (int k = 0; k < S::IDXR; ++k) {
      const int f = flat + k * T;
      if (f < S::IDX && f < lim) {
        const int gi = r[k];
        sI[b * S::IDX + f] = gi;
        const int e = f / n3, l = f - e * n3;
        float* dst = sX + b * NE * S::XE + e * S::XE + (l / n) * S::XL + (l % n);
        if (gi >= 0)
          cp_async4(dst, x + gi);
        else
          *dst = 0.f;
      }
    }
    cp_async_commit();
  };

  if (flat == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  __syncthreads();
  if (flat == 0) issue_d(g, 0);
  {
    int r[S::IDXR];
    load_idx(g, r);
    gather(g, 0, r);
  }
  uint32_t ph0 = 0u, ph1 = 0u;  // parity of the next wait on buffer 0 / 1
  int cur = 0;
  for (; g < G; g += gridDim.x) {
    const int gn = g + gridDim.x;
    const bool has_next = gn < G;
    const int nxt = cur ^ 1;
    if (has_next && flat == 0) issue_d(gn, nxt);
    int r[S::IDXR];
    if (has_next) load_idx(gn, r);
    cp_async_wait_all();
    __syncthreads();
    const int64_t e0 = (int64_t)g * NE;
    const int ne = (int)((E - e0) < NE ? (E - e0) : NE);
    const bool live = el < ne;
    {
      int e, ln;
      stage_item<FLAT, n * n, TPE>(tid, el, e, ln);
      f32_stage1<P, Q, DIFF>(ln, e < ne, sX + cur * NE * S::XE + e * S::XE, sS1 + e * S::W1);
    }
    __syncthreads();
    {
      int e, ln;
      stage_item<FLAT, Q * n, TPE>(tid, el, e, ln);
      f32_stage2<P, Q, DIFF>(ln, e < ne, sS1 + e * S::W1, sS2 + e * S::W2);
    }
    if (has_next) gather(gn, nxt, r);
    const uint32_t pc = cur ? ph1 : ph0, pn = cur ? ph0 : ph1;
    const bool ok = mbar_wait_bounded(&mbar[cur], pc, c_first_wait_limit);
    if (cur) ph1 ^= 1u; else ph0 ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (flat == 0) {
        atomicOr(err, 1);
        mbar_wait_bounded(&mbar[cur], pc);  // let the copies in flight finish before exiting
        if (has_next) mbar_wait_bounded(&mbar[nxt], pn);
      }
      cp_async_wait_all();
      return;
    }
    f32_stage3<P, Q, DIFF>(tid, live, S2, sD + cur * NE * S::DELEM + el * S::DELEM + tid);
    __syncthreads();
    {
      int e, ln;
      stage_item<FLAT, Q * n, TPE>(tid, el, e, ln);
      f32_stage2t<P, Q, DIFF>(ln, e < ne, sS2 + e * S::W2, sS1 + e * S::W1);
    }
    __syncthreads();
    {
      int e, ln;
      stage_item<FLAT, n * n, TPE>(tid, el, e, ln);
      f32_stage1t<P, Q, DIFF>(ln, e < ne, sS1 + e * S::W1, sI + cur * S::IDX + e * n3, x, y);
    }
    __syncthreads();
    cur = nxt;
  }
}

// FP64 D [e][comp][q^3] -> padded FP32 D [e][comp][DSTRIDE]
__global__ void pad_to_f32(int64_t E, int ncomp, int q3, int dstride, const double* __restrict__ qd,
                           float* __restrict__ qd32) {
  const int64_t total = E * ncomp * (int64_t)dstride;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ec = t / dstride;
    const int k = (int)(t - ec * dstride);
    qd32[t] = k < q3 ? (float)qd[ec * q3 + k] : 0.f;
  }
}

}  // namespace fepa
