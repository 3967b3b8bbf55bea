// FP32 fused partial-assembly action for the mixed-precision solve (the operator
// y = G^T B^T D B G x of Fig. fig_feod, arXiv 2402.15940), built for an HBM-bound
// kernel on sm_103a:
//   * each thread block owns NE consecutive elements; at entry one thread issues a
//     single TMA bulk copy (cp.async.bulk, completion on an mbarrier) of the block's
//     D data -- contiguous in HBM -- into shared memory, which overlaps the gather
//     and the first two contraction stages;
//   * the 1D tables live in __constant__ memory at compile-time offsets, so with the
//     loops unrolled they are free FMA operands;
//   * every stage is register-blocked: a thread loads one line of its element once
//     and produces all outputs of that line (stage 3, the pointwise D and the
//     transposed stage 3 stay in registers per (i,j) column, as in the FP64 kernel).
// D here is the FP32 copy with each component padded to a multiple of 4 floats, so
// every element's block is a multiple of 16 bytes (the bulk-copy granularity).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pa_kernels.cuh"

namespace fepa {

// tables of every compiled (P, Q): slot ((P-1)*2 + (Q-P-1)) holds B then G, 100 floats each
constexpr int TAB_SLOT = 200;
constexpr int TAB_SLOTS = 16;
__constant__ float c_tab32[TAB_SLOT * TAB_SLOTS];

template <int P, int Q>
struct Tab32 {
  static_assert(Q == P + 1 || Q == P + 2, "compiled q");
  static constexpr int OFF = ((P - 1) * 2 + (Q - P - 1)) * TAB_SLOT;
  static __device__ __forceinline__ float B(int i, int a) { return c_tab32[OFF + i * (P + 1) + a]; }
  static __device__ __forceinline__ float G(int i, int a) { return c_tab32[OFF + 100 + i * (P + 1) + a]; }
};

// Launch shape of one compiled variant.  STAGE_D: D of the block's elements is brought
// into shared memory by one TMA bulk copy (true) or read by each thread straight from
// HBM in stage 3 (false: a smaller block footprint, so more warps per SM).  NE_DIV
// divides the default number of elements per block.
template <int P, int Q, bool DIFF, bool STAGE_D = true, int NE_DIV = 1>
struct TmaShape {
  static constexpr int N = P + 1;
  static constexpr int NC = DIFF ? 6 : 1;
  static constexpr int Q3 = Q * Q * Q;
  static constexpr int DSTRIDE = (Q3 + 3) & ~3;  // floats per stored component (16-byte multiple)
  static constexpr int DELEM = NC * DSTRIDE;     // floats of D per element
  static constexpr int NC1 = DIFF ? 2 : 1;
  static constexpr int NC2 = DIFF ? 3 : 1;
  static constexpr int WORK = N * N * N + NC1 * N * N * Q + NC2 * N * Q * Q;  // stage buffers, floats
  static constexpr int TPE = Q * Q;
  static constexpr int NE0 = (256 / TPE) > 0 ? (256 / TPE) : 1;
  static constexpr int NE = (NE0 / NE_DIV) > 0 ? (NE0 / NE_DIV) : 1;
  static constexpr int SMEM = 16 + NE * ((STAGE_D ? DELEM : 0) + WORK) * 4;
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

// Bounded wait for phase 0 of the barrier: false if it did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, 0)) return true;
  return false;
}

template <int P, int Q, bool DIFF, bool STAGE_D, int NE_DIV>
__global__ void __launch_bounds__(TmaShape<P, Q, DIFF, STAGE_D, NE_DIV>::TPE * TmaShape<P, Q, DIFF, STAGE_D, NE_DIV>::NE)
pa_apply_f32_tma(int E, const int* __restrict__ gmap, const float* __restrict__ qd32, const float* __restrict__ x,
                 float* __restrict__ y, const int* __restrict__ skip, int* __restrict__ err) {
  using S = TmaShape<P, Q, DIFF, STAGE_D, NE_DIV>;
  using T = Tab32<P, Q>;
  constexpr int n = S::N, TPE = S::TPE, NE = S::NE;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_tma[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_tma);
  float* sD = reinterpret_cast<float*>(smem_tma + 16);
  float* sW = sD + (STAGE_D ? NE * S::DELEM : 0);
  const int tid = threadIdx.x, el = threadIdx.y;
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int ne = (int)((E - e0) < NE ? (E - e0) : NE);
  if (STAGE_D && tid == 0 && el == 0) {
    mbar_init(mbar, 1);
    const uint32_t bytes = (uint32_t)ne * S::DELEM * 4u;
    mbar_expect_tx(mbar, bytes);
    bulk_copy_g2s(sD, qd32 + e0 * S::DELEM, bytes, mbar);
  }
  const bool live = el < ne;
  float* sX = sW + el * S::WORK;
  float* S1 = sX + n * n * n;
  float* S2 = S1 + S::NC1 * n * n * Q;
  const int* g = gmap + (e0 + el) * (n * n * n);
  if (live)
    for (int l = tid; l < n * n * n; l += TPE) {
      const int gi = g[l];
      sX[l] = gi >= 0 ? x[gi] : 0.f;
    }
  __syncthreads();

  // stage 1 (x): line (b,c) -> S1[m][c][b][i] for all i
  if (live && tid < n * n) {
    float xv[n];
#pragma unroll
    for (int a = 0; a < n; ++a) xv[a] = sX[tid * n + a];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float sb = 0.f, sg = 0.f;
#pragma unroll
      for (int a = 0; a < n; ++a) {
        sb = fmaf(T::B(i, a), xv[a], sb);
        if (DIFF) sg = fmaf(T::G(i, a), xv[a], sg);
      }
      S1[tid * Q + i] = sb;
      if (DIFF) S1[n * n * Q + tid * Q + i] = sg;
    }
  }
  __syncthreads();

  // stage 2 (y): line (i,c) -> S2[m][c][j][i] for all j
  //   DIFF: m=0 (x:G,y:B), m=1 (x:B,y:G), m=2 (x:B,y:B); mass: m=0 (B,B)
  if (live && tid < Q * n) {
    const int i = tid % Q, c = tid / Q;
    float vb[n], vg[n];
#pragma unroll
    for (int b = 0; b < n; ++b) {
      vb[b] = S1[i + Q * (b + n * c)];
      if (DIFF) vg[b] = S1[n * n * Q + i + Q * (b + n * c)];
    }
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
      const int o = c * Q * Q + j * Q + i;
      if (DIFF) {
        S2[o] = gb;
        S2[n * Q * Q + o] = bg;
        S2[2 * n * Q * Q + o] = bb;
      } else {
        S2[o] = bb;
      }
    }
  }

  if (STAGE_D) {
    // D must have landed before stage 3; every thread observes the barrier (bounded)
    const bool ok = mbar_wait_bounded(mbar);
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

  // stage 3 (z) + D + stage 3^T, one (i,j) column per thread, in registers
  if (live) {
    float c0[n], c1[n], c2[n], a0[n], a1[n], a2[n];
#pragma unroll
    for (int c = 0; c < n; ++c) {
      c0[c] = S2[c * Q * Q + tid];
      if (DIFF) {
        c1[c] = S2[n * Q * Q + c * Q * Q + tid];
        c2[c] = S2[2 * n * Q * Q + c * Q * Q + tid];
      }
      a0[c] = 0.f;
      if (DIFF) a1[c] = a2[c] = 0.f;
    }
    const float* dE = (STAGE_D ? sD + el * S::DELEM : qd32 + (e0 + el) * S::DELEM) + tid;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      if (DIFF) {
        float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
        for (int c = 0; c < n; ++c) {
          u0 = fmaf(T::B(k, c), c0[c], u0);
          u1 = fmaf(T::B(k, c), c1[c], u1);
          u2 = fmaf(T::G(k, c), c2[c], u2);
        }
        const float* dk = dE + k * Q * Q;
        const float d00 = dk[0], d01 = dk[S::DSTRIDE], d02 = dk[2 * S::DSTRIDE], d11 = dk[3 * S::DSTRIDE],
                    d12 = dk[4 * S::DSTRIDE], d22 = dk[5 * S::DSTRIDE];
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
        const float v = dE[k * Q * Q] * u;
#pragma unroll
        for (int c = 0; c < n; ++c) a0[c] = fmaf(T::B(k, c), v, a0[c]);
      }
    }
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

  // stage 2^T (y): line (i,c) -> S1[0][c][b][i] = sum_j B[j][b] A0,
  //                               S1[1][c][b][i] = sum_j G[j][b] A1 + B[j][b] A2
  if (live && tid < Q * n) {
    const int i = tid % Q, c = tid / Q;
    float v0[Q], v1[Q], v2[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      v0[j] = S2[c * Q * Q + j * Q + i];
      if (DIFF) {
        v1[j] = S2[n * Q * Q + c * Q * Q + j * Q + i];
        v2[j] = S2[2 * n * Q * Q + c * Q * Q + j * Q + i];
      }
    }
#pragma unroll
    for (int b = 0; b < n; ++b) {
      float t0 = 0.f, t1 = 0.f;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        t0 = fmaf(T::B(j, b), v0[j], t0);
        if (DIFF) t1 = fmaf(T::G(j, b), v1[j], fmaf(T::B(j, b), v2[j], t1));
      }
      S1[i + Q * (b + n * c)] = t0;
      if (DIFF) S1[n * n * Q + i + Q * (b + n * c)] = t1;
    }
  }
  __syncthreads();

  // stage 1^T (x): line (b,c) -> y[g(a,b,c)] += sum_i G[i][a] T0 + B[i][a] T1
  if (live && tid < n * n) {
    float t0[Q], t1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      t0[i] = S1[tid * Q + i];
      if (DIFF) t1[i] = S1[n * n * Q + tid * Q + i];
    }
#pragma unroll
    for (int a = 0; a < n; ++a) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (DIFF)
          s = fmaf(T::G(i, a), t0[i], fmaf(T::B(i, a), t1[i], s));
        else
          s = fmaf(T::B(i, a), t0[i], s);
      }
      const int gi = g[a + n * tid];
      if (gi >= 0) {
        atomicAdd(y + gi, s);
      } else if (!((~gi) & ESS_SKIP)) {
        atomicAdd(y + (~gi), x[~gi]);
      }
    }
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
