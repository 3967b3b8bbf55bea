// C-ABI of the partial-assembly library (declarations and conventions: include/fepa.h).
//
// Host side: validates arguments, builds the 1D tables, owns device arrays, dispatches
// the compiled (p, q, form) kernel instances, and drives CG either through a CUDA graph
// whose while-node repeats one iteration until a device-side flag says stop, or (stream
// mode) through short host-driven chunks of the same kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/fepa.h"
#include "basis1d.hpp"
#include "hex_mesh.hpp"
#include "cg_kernels.cuh"
#include "pa_kernels.cuh"
#include "pa_tma_f32.cuh"
#include "pa_df64.cuh"
#include "geom_df.cuh"
#include "batch_kernels.cuh"
#include "mg_kernels.cuh"

using namespace fepa;

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(call)                                                                               \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail(FEPA_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                          \
  } while (0)

// counts the launch, then checks it
#define LAUNCH_CHECK()                                                                               \
  do {                                                                                               \
    g_launches.fetch_add(1);                                                                         \
    cudaError_t e_ = cudaGetLastError();                                                             \
    if (e_ != cudaSuccess) return fail(FEPA_ERR_CUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                          \
  } while (0)

// checks a launch without counting it (loop bodies, counted by iterations run)
#define BODY_CHECK()                                                                                 \
  do {                                                                                               \
    cudaError_t e_ = cudaGetLastError();                                                             \
    if (e_ != cudaSuccess) return fail(FEPA_ERR_CUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                          \
  } while (0)

#define TRY(call)                   \
  do {                              \
    int rc_ = (call);               \
    if (rc_ != FEPA_OK) return rc_; \
  } while (0)

inline int grid_for(int64_t work, int threads, int cap) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// ---------------------------------------------------------------------------
// compiled kernel instances, indexed by p (1..8), q - p - 1 (0, 1), form (0, 1)
// ---------------------------------------------------------------------------
template <typename R>
using ApplyFn = void (*)(int, const int*, const R*, const R*, const R*, const R*, R*, const int*, const int*,
                         const int*);
using Apply32Fn = void (*)(int, const int*, const float*, const float*, float*, const int*, const int*, const int*,
                           int*, double*);

constexpr int N32_VARIANTS = 4;  // (staged D, NE), (direct D, NE), (direct D, NE/2), persistent pipeline
// FP64 pipe (DFMA), double-float on the FP32 pipe, double-float in half-size blocks
constexpr int N64_VARIANTS = 3;
constexpr bool df_variant(int v) { return v == 1 || v == 2; }
using ApplyDfFn = void (*)(int, const int*, const float2*, const double*, double*, const int*, const int*,
                          const int*, int);

struct Apply32Variant {
  Apply32Fn fn;
  int smem, ne, threads_y;
  bool persistent;
};

struct KernelSet {
  ApplyFn<double> apply;
  ApplyDfFn apply_df[2];  // double-float action, full- and half-size blocks (FP64 variants 1, 2)
  int df_smem[2], df_ne[2];
  void (*diag_df)(int, const int*, const float2*, double*);
  int diag_df_smem, diag_df_ne;
  void (*rhs_df)(int64_t, int, int, const int*, const float2*, const int*, const double*, double, double, double*);
  int rhs_df_smem, rhs_df_ne;
  Apply32Variant v32[N32_VARIANTS];
  // persistent forms over a work list of element tiles (the batch's iteration loops)
  void (*apply_tiles)(const int2*, const int*, const int*, const int*, const double*, const double*, const double*,
                      const double*, double*, const int*);
  void (*apply_df_tiles[2])(const int2*, const int*, const int*, const int*, const float2*, const double*, double*,
                            const int*, int);
  void (*apply32_tiles[2])(const int2*, const int*, const int*, const int*, const float*, const float*, float*,
                           const int*, int*);  // shapes of variants 1 and 2
  Apply32Fn v32dot[3] = {};  // variants 0-2 built to add (x, A x) into DOT_SLOTS doubles (p >= 3)
  void (*diag)(int, const int*, const double*, const double*, const double*, double*);
  int apply_smem, apply_tpe, apply_ne;
  int d32_stride;
  int diag_smem;
};

template <int P, int Q, bool DIFF>
KernelSet make_set() {
  KernelSet k;
  k.apply = pa_apply<double, P, Q, DIFF>;
  k.apply_df[0] = pa_apply_df<P, Q, DIFF, 1>;
  k.apply_df[1] = pa_apply_df<P, Q, DIFF, 2>;
  k.df_smem[0] = DfShape<P, Q, DIFF, 1>::SMEM;
  k.df_smem[1] = DfShape<P, Q, DIFF, 2>::SMEM;
  k.df_ne[0] = DfShape<P, Q, DIFF, 1>::NE;
  k.df_ne[1] = DfShape<P, Q, DIFF, 2>::NE;
  k.diag_df = pa_diag_df<P, Q, DIFF>;
  k.diag_df_smem = DiagDfShape<P, Q, DIFF>::SMEM;
  k.diag_df_ne = DiagDfShape<P, Q, DIFF>::NE;
  k.rhs_df = pa_rhs_df<P, Q>;
  k.rhs_df_smem = RhsDfShape<P, Q>::SMEM;
  k.rhs_df_ne = RhsDfShape<P, Q>::NE;
  k.v32[0] = {pa_apply_f32_tma<P, Q, DIFF, true, 1>, TmaShape<P, Q, DIFF, true, 1>::SMEM,
              TmaShape<P, Q, DIFF, true, 1>::NE, TmaShape<P, Q, DIFF, true, 1>::NE, false};
  k.v32[1] = {pa_apply_f32_tma<P, Q, DIFF, false, 1>, TmaShape<P, Q, DIFF, false, 1>::SMEM,
              TmaShape<P, Q, DIFF, false, 1>::NE, TmaShape<P, Q, DIFF, false, 1>::NE, false};
  k.v32[2] = {pa_apply_f32_tma<P, Q, DIFF, false, 2>, TmaShape<P, Q, DIFF, false, 2>::SMEM,
              TmaShape<P, Q, DIFF, false, 2>::NE, TmaShape<P, Q, DIFF, false, 2>::NE, false};
  k.v32[3] = {pa_apply_f32_pipe<P, Q, DIFF>, PipeShape<P, Q, DIFF>::SMEM, PipeShape<P, Q, DIFF>::NE,
              PipeShape<P, Q, DIFF>::NE, true};
  k.apply_tiles = pa_apply_tiles<double, P, Q, DIFF>;
  k.apply_df_tiles[0] = pa_apply_df_tiles<P, Q, DIFF, 1>;
  k.apply_df_tiles[1] = pa_apply_df_tiles<P, Q, DIFF, 2>;
  k.apply32_tiles[0] = pa_apply_f32_tiles<P, Q, DIFF, 1>;
  k.apply32_tiles[1] = pa_apply_f32_tiles<P, Q, DIFF, 2>;
  if constexpr (P >= 3) {
    k.v32dot[0] = pa_apply_f32_tma<P, Q, DIFF, true, 1, 2, (P <= 4), (P <= 3), false, true>;
    k.v32dot[1] = pa_apply_f32_tma<P, Q, DIFF, false, 1, 2, (P <= 4), (P <= 3), false, true>;
    k.v32dot[2] = pa_apply_f32_tma<P, Q, DIFF, false, 2, 2, (P <= 4), (P <= 3), false, true>;
  }

  k.diag = pa_diag_f64<P, Q, DIFF>;
  k.apply_smem = PaShape<double, P, Q, DIFF>::SMEM;
  k.apply_tpe = PaShape<double, P, Q, DIFF>::TPE;
  k.apply_ne = PaShape<double, P, Q, DIFF>::NE;
  k.d32_stride = TmaShape<P, Q, DIFF>::DSTRIDE;
  k.diag_smem = DiagShape<P, Q, DIFF>::SMEM;
  return k;
}

static_assert(FEPA_MAX_ORDER == 8, "the FP32 pair tables (tab32_offset) are laid out for p = 1..8");

template <int P>
void fill_order(KernelSet (&t)[FEPA_MAX_ORDER + 1][2][2]) {
  t[P][0][0] = make_set<P, P + 1, false>();
  t[P][0][1] = make_set<P, P + 1, true>();
  t[P][1][0] = make_set<P, P + 2, false>();
  t[P][1][1] = make_set<P, P + 2, true>();
}

struct KernelTable {
  KernelSet t[FEPA_MAX_ORDER + 1][2][2];
  KernelTable() {
    fill_order<1>(t);
    fill_order<2>(t);
    fill_order<3>(t);
    fill_order<4>(t);
    fill_order<5>(t);
    fill_order<6>(t);
    fill_order<7>(t);
    fill_order<8>(t);
  }
};

const KernelTable& kernels() {
  static KernelTable table;
  return table;
}

// (hi, lo) float pairs of the FP64 1D tables for the double-float action, into the
// constant-memory slot of (p, q)
int upload_df_tables(int p, int q, const std::vector<double>& Bh, const std::vector<double>& Gh, cudaStream_t s) {
  const int n = p + 1, qh = (q + 1) / 2, nh = (n + 1) / 2;
  // the pair layout of TabDf: (hi pair, lo pair) per entry; rows then columns, B then G
  std::vector<float2> tdf;
  tdf.reserve(2 * tab32_slot_pairs(p, q));
  auto put_pair = [&](double a, double b) {
    const float ah = (float)a, bh = (float)b;
    tdf.push_back(make_float2(ah, bh));
    tdf.push_back(make_float2((float)(a - (double)ah), (float)(b - (double)bh)));
  };
  for (const std::vector<double>* T : {&Bh, &Gh})
    for (int kp = 0; kp < qh; ++kp)
      for (int a = 0; a < n; ++a) put_pair((*T)[2 * kp * n + a], 2 * kp + 1 < q ? (*T)[(2 * kp + 1) * n + a] : 0.0);
  for (const std::vector<double>* T : {&Bh, &Gh})
    for (int k = 0; k < q; ++k)
      for (int ap = 0; ap < nh; ++ap) put_pair((*T)[k * n + 2 * ap], 2 * ap + 1 < n ? (*T)[k * n + 2 * ap + 1] : 0.0);
  CUDA_TRY(cudaMemcpyToSymbolAsync(c_tabdf, tdf.data(), tdf.size() * sizeof(float2),
                                   2 * (size_t)tab32_offset(p, q) * sizeof(float2), cudaMemcpyHostToDevice, s));
  if (q != p + 2) return FEPA_OK;
  // even/odd tables of B, G (q x n) and B^T, G^T (n x q) for the double-float action
  // entry k of matrix mat: a hi pair then a lo pair; half 0 (x) or 1 (y) of the pair
  std::vector<float2> teo(4 * EO_MAT * 2, make_float2(0.f, 0.f));
  auto put = [&](int mat, int k, int half, double v) {
    const float h = (float)v, l = (float)(v - (double)h);
    float2& ph = teo[2 * (mat * EO_MAT + k)];
    float2& pl = teo[2 * (mat * EO_MAT + k) + 1];
    (half ? ph.y : ph.x) = h;
    (half ? pl.y : pl.x) = l;
  };
  for (int mat = 0; mat < 4; ++mat) {
    const std::vector<double>& M = (mat % 2 == 0) ? Bh : Gh;
    const int NO = mat < 2 ? q : n, NI = mat < 2 ? n : q, HO = NO / 2, HI = NI / 2;
    const double S = (mat % 2 == 0) ? 1.0 : -1.0;
    auto m = [&](int o, int i) { return mat < 2 ? M[o * n + i] : M[i * n + o]; };  // B(q, a) at q*n + a
    double scale = 0.0;
    for (int o = 0; o < NO; ++o)
      for (int i = 0; i < NI; ++i) scale = std::max(scale, fabs(m(o, i)));
    for (int o = 0; o < NO; ++o)
      for (int i = 0; i < NI; ++i)
        if (fabs(m(NO - 1 - o, NI - 1 - i) - S * m(o, i)) > 1e-13 * scale)
          return fail(FEPA_ERR_CUDA, "1D tables of p=%d q=%d are not symmetric", p, q);
    for (int o = 0; o < HO; ++o)
      for (int i = 0; i < HI; ++i) {
        put(mat, o * HI + i, 0, 0.5 * (m(o, i) + m(o, NI - 1 - i)));
        put(mat, o * HI + i, 1, 0.5 * (m(o, i) - m(o, NI - 1 - i)));
      }
    if (NI % 2)
      for (int o = 0; o < HO; ++o) put(mat, HO * HI + o, 0, m(o, HI));
    if (NO % 2)
      for (int i = 0; i <= HI && i < NI; ++i) put(mat, HO * HI + HO + i, 0, m(HO, i));
  }
  CUDA_TRY(cudaMemcpyToSymbolAsync(c_tabeo, teo.data(), teo.size() * sizeof(float2),
                                   (size_t)(p - 1) * 4 * EO_MAT * 2 * sizeof(float2), cudaMemcpyHostToDevice, s));
  return FEPA_OK;
}

// Gauss points and weights of q as (hi, lo) float pairs (long double on the host), into
// the constant-memory slot of q for the double-float geometry
int upload_gauss_df(int q, const std::vector<long double>& x, const std::vector<long double>& w, cudaStream_t s) {
  std::vector<float> t(2 * GQ_MAX * 2, 0.f);
  for (int i = 0; i < q; ++i) {
    const float xh = (float)x[i], wh = (float)w[i];
    t[2 * i] = xh;
    t[2 * i + 1] = (float)(x[i] - (long double)xh);
    t[2 * (GQ_MAX + i)] = wh;
    t[2 * (GQ_MAX + i) + 1] = (float)(w[i] - (long double)wh);
  }
  CUDA_TRY(cudaMemcpyToSymbolAsync(c_gauss_df, t.data(), t.size() * sizeof(float),
                                   (size_t)q * 2 * GQ_MAX * 2 * sizeof(float), cudaMemcpyHostToDevice, s));
  return FEPA_OK;
}

int allow_smem(const void* fn, int bytes) {
  if (bytes > 48 * 1024) CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return FEPA_OK;
}

// One CG loop (FP64 or FP32 inner): work vectors, device scalars, and its cached graph.
struct CgLoop {
  void* x = nullptr;  // iterate (FP32 loops own it; the FP64 loop iterates in a copy)
  void *r = nullptr, *d = nullptr, *h = nullptr;
  void* invd = nullptr;  // 1/diag in the loop's precision
  CgState* st = nullptr;
  double* partials = nullptr;
  int red_blocks = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_key = -1;  // preconditioner and kernel variants the cached graph was captured with
  double* dh_slots = nullptr;  // FP32 loop: (d, h) accumulated by the fused action
  int kernels_per_iter = 4;    // launches per iteration of the body last built (stream mode)
  int graph_kernels_per_iter = 4;  // launches per iteration of the cached graph's body
};

}  // namespace

struct fepa_op {
  int nx, ny, nz, p, q, n, form;  // nx, ny, nz: structured grid (unused when hex)
  int64_t E, N;
  int64_t nverts;                 // vertices of the mesh
  bool hex = false;               // built from element connectivity (fepa_op_create_hex)
  int* econn = nullptr;           // hex: device [E][8] corner vertex ids
  std::vector<int32_t> conn_host; // hex: the connectivity (for derived ops, e.g. multigrid levels)
  std::vector<int32_t> bdr_host;  // hex: DOFs on faces held by one element, ascending
  int device;
  int cg_mode = FEPA_CG_GRAPH;
  int fuse_dot = 1;  // FP32 CG: (d, h) from the action kernel where it has that build
  double* dot_slots = nullptr;  // fepa_op_apply_f32_dot's accumulators
  cudaStream_t stream;
  cudaStream_t cap_stream;  // private stream used only to capture graphs
  KernelSet ks;
  std::vector<float> B32h, G32h;
  std::vector<double> verts_host;  // host copy of the vertex grid (for derived ops, e.g. multigrid levels)
  // device arrays owned by the op
  double* verts = nullptr;
  float2* verts_df = nullptr;  // the vertices as (hi, lo) float pairs (double-float geometry)
  int* gmap = nullptr;
  double* qd = nullptr;
  double* B = nullptr;
  double* G = nullptr;
  double* pts = nullptr;
  double* wts = nullptr;
  int* ess = nullptr;
  int64_t ess_count = 0;
  int* flag = nullptr;  // device ints: [0] mesh check bits, [1] largest exponent of D
  int dexp = 0;         // largest binary exponent of D (from the last geometry pass)
  // FP32 operator data (built on first use): padded FP32 D; tables in constant memory
  float* qd32 = nullptr;
  bool qd32_valid = false;
  // double-float action data (built when that variant is in use): D as (hi, lo) floats
  float2* qddf = nullptr;
  bool qddf_valid = false;
  int v32 = -1;        // FP32 kernel variant in use (-1: not chosen yet)
  int v32_grid[4] = {0, 0, 0, 0};  // launch grid per variant (persistent: SMs x resident blocks)
  int v32_forced = -1; // variant set by the caller (-1: autotune)
  int v64 = -1;        // FP64 action variant in use (-1: not chosen yet)
  int v64_forced = -1; // variant set by the caller (-1: autotune)
  int* err = nullptr;  // device word set by kernels whose bounded waits expired
  // CG workspace (allocated on first solve)
  double* inv_diag = nullptr;
  bool inv_diag_valid = false;
  double* xw = nullptr;
  double *bw = nullptr, *xio = nullptr;  // host-buffer solves
  CgLoop cg64, cg32;
  // refinement: FP64 residual, its scalars
  double* h64 = nullptr;
  CgState* st_ref = nullptr;
  double* partials_ref = nullptr;
  bool inv32_valid = false;
  CgState* st_host = nullptr;  // pinned
  int* st_host_flag = nullptr;  // pinned
  // resumable solve (fepa_solver_*)
  int sv_kind = -1, sv_phase = 0, sv_precond = 0, sv_outer = 0, sv_inner_total = 0, sv_maxit = 0, sv_max_outer = 0;
  int sv_status = 0;
  int sv_seen_iter = 0;  // iterations already counted in the launch counter
  double sv_rtol = 0.0, sv_inner_rtol = 0.0, sv_rel = 0.0;
  double sv_rscale = 1.0;  // power of two the current inner solve's residual was scaled by
  const double* sv_b = nullptr;
  double* sv_x = nullptr;
  cudaEvent_t sv_event = nullptr;
};

namespace {

void free_loop(CgLoop& L) {
  if (L.exec) cudaGraphExecDestroy(L.exec);
  if (L.graph) cudaGraphDestroy(L.graph);
  for (void* p : {L.x, L.r, L.d, L.h, L.invd, (void*)L.st, (void*)L.partials, (void*)L.dh_slots})
    if (p) cudaFree(p);
  L = CgLoop();
}

void free_op(fepa_op* op) {
  if (!op) return;
  cudaStreamSynchronize(op->stream);
  free_loop(op->cg64);
  free_loop(op->cg32);
  for (void* p : {(void*)op->verts, (void*)op->verts_df, (void*)op->econn, (void*)op->gmap, (void*)op->qd, (void*)op->B, (void*)op->G, (void*)op->pts,
                  (void*)op->wts, (void*)op->ess, (void*)op->flag, (void*)op->qd32, (void*)op->qddf, (void*)op->err,
                  (void*)op->inv_diag, (void*)op->xw, (void*)op->bw, (void*)op->xio, (void*)op->h64,
                  (void*)op->st_ref, (void*)op->partials_ref, (void*)op->dot_slots})
    if (p) cudaFree(p);
  if (op->st_host) cudaFreeHost(op->st_host);
  if (op->st_host_flag) cudaFreeHost(op->st_host_flag);
  if (op->sv_event) cudaEventDestroy(op->sv_event);
  if (op->cap_stream) cudaStreamDestroy(op->cap_stream);
  delete op;
}

template <typename T>
int dalloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(FEPA_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
  }
  return FEPA_OK;
}

// y += A x in FP64 with variant v (launch only; not counted)
int launch_apply64_variant(fepa_op* op, int v, const double* x, double* y, const int* skip, cudaStream_t s) {
  const KernelSet& k = op->ks;
  if (df_variant(v)) {
    const int sh = v - 1;  // block shape: full or half
    const int grid = (int)((op->E + k.df_ne[sh] - 1) / k.df_ne[sh]);
    k.apply_df[sh]<<<grid, dim3(k.apply_tpe, k.df_ne[sh]), k.df_smem[sh], s>>>((int)op->E, op->gmap, op->qddf, x, y,
                                                                               skip, nullptr, nullptr, op->dexp);
  } else {
    const int grid = (int)((op->E + k.apply_ne - 1) / k.apply_ne);
    k.apply<<<grid, dim3(k.apply_tpe, k.apply_ne), k.apply_smem, s>>>((int)op->E, op->gmap, op->qd, op->B, op->G, x,
                                                                      y, skip, nullptr, nullptr);
  }
  BODY_CHECK();
  return FEPA_OK;
}

int prepare_f64(fepa_op* op);

// y += A x in FP64 without choosing a variant (no timing, no allocation): the chosen or
// forced variant, else the DFMA kernel (counted)
int launch_apply_untuned(fepa_op* op, const double* x, double* y, const int* skip, cudaStream_t s) {
  int v = op->v64 >= 0 ? op->v64 : (op->v64_forced >= 0 ? op->v64_forced : 0);
  if (df_variant(v) && !op->qddf_valid) v = 0;  // its D copy would need an allocation
  TRY(launch_apply64_variant(op, v, x, y, skip, s));
  g_launches.fetch_add(1);
  return FEPA_OK;
}

// y += A x in FP64 (launch only; counted)
int launch_apply(fepa_op* op, const double* x, double* y, const int* skip, cudaStream_t s) {
  TRY(prepare_f64(op));
  TRY(launch_apply64_variant(op, op->v64, x, y, skip, s));
  g_launches.fetch_add(1);
  return FEPA_OK;
}

// whether FP32 variant v has a build that also adds (x, A x) into DOT_SLOTS doubles
bool has_dot_build(const fepa_op* op, int v) { return v >= 0 && v < 3 && op->ks.v32dot[v]; }

// y += A x in FP32 with variant v (launch only; not counted).  dot: also add (x, A x) into
// these DOT_SLOTS doubles (only where fused_dot_ok).
int launch_apply32_variant(fepa_op* op, int v, const float* x, float* y, const int* skip, cudaStream_t s,
                           double* dot = nullptr) {
  const Apply32Variant& k = op->ks.v32[v];
  const int grid = op->v32_grid[v];
  if (grid <= 0) return fail(FEPA_ERR_UNSUPPORTED, "FP32 variant %d cannot run with this shape", v);
  const Apply32Fn fn = dot ? (v < 3 ? op->ks.v32dot[v] : nullptr) : k.fn;
  if (!fn) return fail(FEPA_ERR_UNSUPPORTED, "FP32 variant %d has no fused (x, A x) build", v);
  fn<<<grid, dim3(op->ks.apply_tpe, k.threads_y), k.smem, s>>>((int)op->E, op->gmap, op->qd32, x, y, skip, nullptr,
                                                                nullptr, op->err, dot);
  BODY_CHECK();
  return FEPA_OK;
}

// grid of every variant: one block per group, or SMs x resident blocks (persistent)
int size_variants32(fepa_op* op) {
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->device));
  for (int v = 0; v < N32_VARIANTS; ++v) {
    const Apply32Variant& k = op->ks.v32[v];
    const int64_t groups = (op->E + k.ne - 1) / k.ne;
    if (!k.persistent) {
      op->v32_grid[v] = (int)groups;
      continue;
    }
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, op->ks.apply_tpe * k.threads_y, k.smem));
    const int64_t g = (int64_t)per_sm * sms;
    op->v32_grid[v] = (int)(g < groups ? g : groups);
  }
  return FEPA_OK;
}

int launch_apply32_nocount(fepa_op* op, const float* x, float* y, const int* skip, cudaStream_t s) {
  return launch_apply32_variant(op, op->v32, x, y, skip, s);
}

// (the variant and its data are prepared before any capture: prepare_f64 runs in run_loop)
int launch_apply_nocount(fepa_op* op, const double* x, double* y, const int* skip, cudaStream_t s) {
  return launch_apply64_variant(op, op->v64 < 0 ? 0 : op->v64, x, y, skip, s);
}

int ensure_host_state(fepa_op* op) {
  if (!op->st_host) CUDA_TRY(cudaMallocHost((void**)&op->st_host, sizeof(CgState)));
  return FEPA_OK;
}

template <typename T>
int ensure_loop(fepa_op* op, CgLoop& L, bool own_x) {
  if (L.r) return FEPA_OK;
  T *r, *d, *h, *iv;
  TRY(dalloc(&r, op->N));
  L.r = r;
  TRY(dalloc(&d, op->N));
  L.d = d;
  TRY(dalloc(&h, op->N));
  L.h = h;
  TRY(dalloc(&iv, op->N));
  L.invd = iv;
  if (own_x) {
    T* x;
    TRY(dalloc(&x, op->N));
    L.x = x;
    TRY(dalloc(&L.dh_slots, DOT_SLOTS));
    CUDA_TRY(cudaMemsetAsync(L.dh_slots, 0, DOT_SLOTS * sizeof(double), op->stream));
  }
  TRY(dalloc(&L.st, 1));
  L.red_blocks = grid_for(op->N, RED_THREADS, 148 * 8);
  TRY(dalloc(&L.partials, 3 * (size_t)L.red_blocks));
  CUDA_TRY(cudaMemsetAsync(L.st, 0, sizeof(CgState), op->stream));
  return ensure_host_state(op);
}

// diag(A) into out: in double-float when that is the op's FP64 arithmetic (and its D copy
// is current), else with the FP64 kernel.  prepare: the variant may be chosen (timed)
// and the D copy built here; the allocation-free solve passes false.
int compute_diagonal(fepa_op* op, double* out, cudaStream_t s, bool prepare = true) {
  if (prepare) TRY(prepare_f64(op));
  CUDA_TRY(cudaMemsetAsync(out, 0, op->N * sizeof(double), s));
  const KernelSet& k = op->ks;
  if (df_variant(op->v64) && op->qddf_valid) {
    const int grid = (int)((op->E + k.diag_df_ne - 1) / k.diag_df_ne);
    k.diag_df<<<grid, dim3(op->q * op->q, k.diag_df_ne), k.diag_df_smem, s>>>((int)op->E, op->gmap, op->qddf, out);
  } else {
    k.diag<<<(int)op->E, op->q * op->q, k.diag_smem, s>>>((int)op->E, op->gmap, op->qd, op->B, op->G, out);
  }
  LAUNCH_CHECK();
  return FEPA_OK;
}

// 1/diag(A) in FP64, kept in op->inv_diag until the mesh or the essential set changes
int ensure_inv_diag(fepa_op* op) {
  if (op->inv_diag_valid) return FEPA_OK;
  if (!op->inv_diag) TRY(dalloc(&op->inv_diag, op->N));
  TRY(compute_diagonal(op, op->inv_diag, op->stream));
  reciprocal<<<grid_for(op->N, 256, 148 * 16), 256, 0, op->stream>>>(op->N, op->inv_diag, op->inv_diag);
  LAUNCH_CHECK();
  op->inv_diag_valid = true;
  op->inv32_valid = false;
  return FEPA_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the FP32 kernel's launch shape and of the FP64 arithmetic: the compiled
// variants are timed on the op's own mesh the first time a (device, p, q, form, size
// class) is used in this process; the fastest is cached and reused.  Size classes of E:
// < 1e3, < 1e4, < 1e5, >= 1e5 elements (small meshes are launch-bound, large ones not).
// ---------------------------------------------------------------------------
constexpr int N_SIZE_CLASSES = 4;
std::mutex g_tune_mutex;
int g_tuned[64][FEPA_MAX_ORDER + 1][2][2][N_SIZE_CLASSES];
int g_tuned64[64][FEPA_MAX_ORDER + 1][2][2][N_SIZE_CLASSES];
bool g_tuned_init = false;

int size_class(int64_t E) { return E < 1000 ? 0 : E < 10000 ? 1 : E < 100000 ? 2 : 3; }

void init_tuned() {
  if (g_tuned_init) return;
  for (auto* t : {&g_tuned, &g_tuned64})
    for (auto& a : *t)
      for (auto& b : a)
        for (auto& c : b)
          for (auto& d : c)
            for (int& v : d) v = -1;
  g_tuned_init = true;
}

// Time the launch functions run(v) of the enabled variants v < nvar on stream s: two warm-up
// calls each, then three rounds, each timing 5 calls of every variant in turn; a variant's time
// is its best round, so that a round slowed by other work on the GPU (another stream of a
// serving process, say) does not decide the choice, which is cached for the process.
template <class Run, class Enabled>
int time_rounds(cudaStream_t s, int nvar, Run run, Enabled enabled, int* best) {
  constexpr int ROUNDS = 3, REPS = 5;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(FEPA_ERR_CUDA, "event creation failed");
  }
  std::vector<float> t(nvar, 1e30f);
  int rc = FEPA_OK;
  for (int v = 0; rc == FEPA_OK && v < nvar; ++v)
    for (int w = 0; w < 2 && rc == FEPA_OK && enabled(v); ++w) rc = run(v);
  for (int round = 0; rc == FEPA_OK && round < ROUNDS; ++round)
    for (int v = 0; rc == FEPA_OK && v < nvar; ++v) {
      if (!enabled(v)) continue;
      cudaEventRecord(e0, s);
      for (int r = 0; r < REPS && rc == FEPA_OK; ++r) rc = run(v);
      cudaEventRecord(e1, s);
      if (rc != FEPA_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = fail(FEPA_ERR_CUDA, "autotune timing failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t[v] = std::min(t[v], ms);
    }
  *best = 0;
  for (int v = 0; v < nvar; ++v)
    if (enabled(v) && (!enabled(*best) || t[v] < t[*best])) *best = v;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int time_variants32(fepa_op* op, int* best) {
  cudaStream_t s = op->stream;
  float *x = nullptr, *y = nullptr;
  double* slots = nullptr;
  TRY(dalloc(&x, op->N));
  int rc = dalloc(&y, op->N);
  if (rc == FEPA_OK) rc = dalloc(&slots, DOT_SLOTS);
  if (rc == FEPA_OK && cudaMemsetAsync(slots, 0, DOT_SLOTS * sizeof(double), s) != cudaSuccess)
    rc = fail(FEPA_ERR_CUDA, "memset failed");
  // each variant in the form the FP32 CG loop launches it: its build with (x, A x) fused where
  // it has one (and the op allows it), else the plain action plus the separate dot pass
  auto run = [&](int v) -> int {
    if (op->fuse_dot && has_dot_build(op, v)) {
      g_launches.fetch_add(1);
      return launch_apply32_variant(op, v, x, y, nullptr, s, slots);
    }
    TRY(launch_apply32_variant(op, v, x, y, nullptr, s));
    dot32_slots<<<grid_for(op->N, RED_THREADS, 148 * 8), RED_THREADS, 0, s>>>(op->N, x, y, slots);
    CUDA_TRY(cudaGetLastError());
    g_launches.fetch_add(2);
    return FEPA_OK;
  };
  *best = 0;
  if (rc == FEPA_OK && cudaMemsetAsync(x, 0, op->N * sizeof(float), s) != cudaSuccess)
    rc = fail(FEPA_ERR_CUDA, "memset failed");
  if (rc == FEPA_OK) rc = time_rounds(s, N32_VARIANTS, run, [&](int v) { return op->v32_grid[v] > 0; }, best);
  cudaFree(x);
  if (y) cudaFree(y);
  if (slots) cudaFree(slots);
  return rc;
}

int choose_variant32(fepa_op* op) {
  if (op->v32_forced >= 0) {
    op->v32 = op->v32_forced;
    return FEPA_OK;
  }
  const int dev = op->device < 64 ? op->device : 63;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  init_tuned();
  int& slot = g_tuned[dev][op->p][op->q - op->p - 1][op->form][size_class(op->E)];
  if (slot < 0) {
    int best = 0;
    TRY(time_variants32(op, &best));
    slot = best;
  }
  op->v32 = slot;
  return FEPA_OK;
}

// (hi, lo) copy of D for the double-float action (allocated once, rebuilt after the mesh moves)
int ensure_df(fepa_op* op) {
  if (op->qddf_valid) return FEPA_OK;
  const int64_t count = op->E * (op->form == FEPA_DIFFUSION ? 6 : 1) * (int64_t)op->q * op->q * op->q;
  if (!op->qddf) TRY(dalloc(&op->qddf, count));
  split_to_df<<<grid_for(count, 256, 148 * 32), 256, 0, op->stream>>>(count, op->qd, op->qddf);
  LAUNCH_CHECK();
  op->qddf_valid = true;
  return FEPA_OK;
}

// Time the FP64 action variants on this op (2 warm-up + 5 timed launches each).
int time_variants64(fepa_op* op, int* best) {
  cudaStream_t s = op->stream;
  double *x = nullptr, *y = nullptr;
  TRY(dalloc(&x, op->N));
  int rc = dalloc(&y, op->N);
  *best = 0;
  if (rc == FEPA_OK && cudaMemsetAsync(x, 0, op->N * sizeof(double), s) != cudaSuccess)
    rc = fail(FEPA_ERR_CUDA, "memset failed");
  if (rc == FEPA_OK) rc = ensure_df(op);
  auto run = [&](int v) -> int {
    g_launches.fetch_add(1);
    return launch_apply64_variant(op, v, x, y, nullptr, s);
  };
  if (rc == FEPA_OK) rc = time_rounds(s, N64_VARIANTS, run, [](int) { return true; }, best);
  cudaFree(x);
  if (y) cudaFree(y);
  return rc;
}

// Cached FP64 variant choice for (device, p, q, form), -1 if none yet (caller holds no lock)
int tuned64_lookup(int device, int p, int q, int form, int64_t E) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  init_tuned();
  return g_tuned64[device < 64 ? device : 63][p][q - p - 1][form][size_class(E)];
}

// FP64 action variant: the caller's, else the fastest one measured for this device, p, q
// and form (both meet the FP64 tolerance; timed once per process)
int ensure_v64(fepa_op* op) {
  if (op->v64 >= 0) return FEPA_OK;
  if (op->v64_forced >= 0) {
    op->v64 = op->v64_forced;
    return FEPA_OK;
  }
  const int dev = op->device < 64 ? op->device : 63;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  init_tuned();
  int& slot = g_tuned64[dev][op->p][op->q - op->p - 1][op->form][size_class(op->E)];
  if (slot < 0) {
    int best = 0;
    TRY(time_variants64(op, &best));
    slot = best;
  }
  op->v64 = slot;
  if (!df_variant(op->v64) && op->qddf) {  // the timing built a D copy the chosen kernel does not read
    cudaStreamSynchronize(op->stream);
    cudaFree(op->qddf);
    op->qddf = nullptr;
    op->qddf_valid = false;
  }
  return FEPA_OK;
}

// variant chosen and its data current (call outside graph capture, before launches)
int prepare_f64(fepa_op* op) {
  TRY(ensure_v64(op));
  if (df_variant(op->v64)) TRY(ensure_df(op));
  return FEPA_OK;
}

// FP32 copy of D (each component padded to a 16-byte multiple) and the FP32 1D tables
// (constant memory, slot of this (p, q)) for the mixed-precision operator
int ensure_f32(fepa_op* op) {
  cudaStream_t s = op->stream;
  const int ncomp = op->form == FEPA_DIFFUSION ? 6 : 1;
  const int q3 = op->q * op->q * op->q;
  const int64_t count = op->E * ncomp * (int64_t)op->ks.d32_stride;
  if (!op->qd32) {
    TRY(dalloc(&op->qd32, count));
    CUDA_TRY(upload_tab32(op->p, op->q, op->B32h, op->G32h, s));
    for (int v = 0; v < N32_VARIANTS; ++v) TRY(allow_smem((const void*)op->ks.v32[v].fn, op->ks.v32[v].smem));
    for (int v = 0; v < 3; ++v)
      if (op->ks.v32dot[v]) TRY(allow_smem((const void*)op->ks.v32dot[v], op->ks.v32[v].smem));
    TRY(size_variants32(op));
  }
  if (!op->qd32_valid) {
    pad_to_f32<<<grid_for(count, 256, 148 * 32), 256, 0, s>>>(op->E, ncomp, q3, op->ks.d32_stride, op->qd, op->qd32);
    LAUNCH_CHECK();
    op->qd32_valid = true;
  }
  if (op->v32 < 0) TRY(choose_variant32(op));
  return FEPA_OK;
}

// D from the vertices (double-float geometry kernel), also refreshing the (hi, lo) and
// FP32 copies of D when they exist.  Sets op->flag if a det J <= 0.
// E elements; corners from econn [E][8] if given, else the structured grid of nx x ny
// elements per layer
template <int Q>
void launch_geom_q(int64_t E, int nx, int ny, const int* econn, const float2* vdf, int diffusion, double* qd,
                   float2* qddf, float* qd32, int d32stride, int* bad, int* dexp, cudaStream_t s) {
  using G = GeoShape<Q>;
  const int grid = (int)((E + G::NE - 1) / G::NE);
  geom_df<Q><<<grid, dim3(G::TPE, G::NE), 0, s>>>(E, nx, ny, econn, vdf, diffusion, qd, qddf, qd32, d32stride, bad,
                                                   dexp);
}

// the geometry kernel of q (2..10); false if q has none.  bad[0]: flag bits (1: det J <= 0,
// 2: outside the double-float set-up's range); dexp (may be null): raised to the largest
// exponent of D
bool launch_geom(int q, int64_t E, int nx, int ny, const int* econn, const float2* vdf, int diffusion, double* qd,
                 float2* qddf, float* qd32, int d32stride, int* bad, int* dexp, cudaStream_t s) {
#define GEOM_CASE(Q) \
  case Q: launch_geom_q<Q>(E, nx, ny, econn, vdf, diffusion, qd, qddf, qd32, d32stride, bad, dexp, s); return true;
  switch (q) {
    GEOM_CASE(2) GEOM_CASE(3) GEOM_CASE(4) GEOM_CASE(5) GEOM_CASE(6) GEOM_CASE(7) GEOM_CASE(8) GEOM_CASE(9)
    GEOM_CASE(10)
    default: return false;
  }
#undef GEOM_CASE
}

int compute_geometry(fepa_op* op) {
  cudaStream_t s = op->stream;
  const int64_t nv3 = 3 * op->nverts;
  if (!op->verts_df) TRY(dalloc(&op->verts_df, nv3));
  split_pairs<<<grid_for(nv3, 256, 148 * 8), 256, 0, s>>>(nv3, op->verts, op->verts_df);
  LAUNCH_CHECK();
  CUDA_TRY(cudaMemsetAsync(op->flag + 1, 0x80, sizeof(int), s));  // D's largest exponent: from -inf
  if (!launch_geom(op->q, op->E, op->nx, op->ny, op->econn, op->verts_df, op->form == FEPA_DIFFUSION, op->qd,
                   op->qddf, op->qd32, op->ks.d32_stride, op->flag, op->flag + 1, s))
    return fail(FEPA_ERR_UNSUPPORTED, "q1d %d has no geometry kernel", op->q);
  LAUNCH_CHECK();
  op->qddf_valid = op->qddf != nullptr;
  op->qd32_valid = op->qd32 != nullptr;
  return FEPA_OK;
}

// After the geometry kernel: FEPA_ERR_MESH for det J <= 0, FEPA_ERR_UNSUPPORTED outside the
// double-float set-up's range; records the largest exponent of D for the action's range test.
int read_mesh_flags(fepa_op* op) {
  CUDA_TRY(cudaMemcpyAsync(op->st_host_flag, op->flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, op->stream));
  CUDA_TRY(cudaStreamSynchronize(op->stream));
  const int bits = op->st_host_flag[0];
  op->dexp = op->st_host_flag[1];
  if (bits & 1) return fail(FEPA_ERR_MESH, "non-positive Jacobian determinant at a quadrature point");
  if (bits & 2)
    return fail(FEPA_ERR_UNSUPPORTED, "an element lies outside the range of the double-float set-up (extent >= 2^-20, "
                                      "|coordinates| <= 2^20 and <= 2^10 x extent): translate or rescale the mesh");
  return FEPA_OK;
}

// FEPA_ERR_TIMEOUT if a kernel of this op gave up a bounded wait since the last check
// (checked at sync points); the word is cleared once read, so each expiry is reported once
int check_err(fepa_op* op) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, op->err, sizeof(int), cudaMemcpyDeviceToHost, op->stream));
  CUDA_TRY(cudaStreamSynchronize(op->stream));
  if (h) {
    CUDA_TRY(cudaMemsetAsync(op->err, 0, sizeof(int), op->stream));
    return fail(FEPA_ERR_TIMEOUT, "a kernel's bounded wait for its staged data expired");
  }
  return FEPA_OK;
}

// ---------------------------------------------------------------------------
// CG loop bodies: one iteration = apply, (d,h), update, direction
// ---------------------------------------------------------------------------
int body64(fepa_op* op, CgLoop& L, const double* invd, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
  const int rb = L.red_blocks;
  double *x = op->xw, *r = (double*)L.r, *d = (double*)L.d, *h = (double*)L.h;
  TRY(launch_apply_nocount(op, d, h, &L.st->done, s));
  cg_dot_dh<<<rb, RED_THREADS, 0, s>>>(op->N, d, h, L.st, L.partials);
  BODY_CHECK();
  cg_update_r<<<rb, RED_THREADS, 0, s>>>(op->N, r, h, invd, L.st, L.partials);
  BODY_CHECK();
  cg_direction_x<<<rb, RED_THREADS, 0, s>>>(op->N, r, d, h, invd, x, L.st, cond, use_cond);
  BODY_CHECK();
  return FEPA_OK;
}

// the final step's x update of a finished FP64 loop (body64 advances x in its direction kernel)
int flush64(fepa_op* op, CgLoop& L, cudaStream_t s) {
  cg_flush64<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, op->xw, (const double*)L.d, L.st);
  LAUNCH_CHECK();
  return FEPA_OK;
}

// FP32 loop: (d, h) comes out of the action kernel itself (no separate pass over d and h)
// when the chosen variant has that build and the op allows it
bool fused_dot_ok(const fepa_op* op) { return op->fuse_dot && has_dot_build(op, op->v32); }

int body32(fepa_op* op, CgLoop& L, const float* invd, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
  const int rb = L.red_blocks;
  float *x = (float*)L.x, *r = (float*)L.r, *d = (float*)L.d, *h = (float*)L.h;
  double* slots = fused_dot_ok(op) ? L.dh_slots : nullptr;
  L.kernels_per_iter = slots ? 3 : 4;
  TRY(launch_apply32_variant(op, op->v32, d, h, &L.st->done, s, slots));
  if (!slots) {
    cg32_dot_dh<<<rb, RED_THREADS, 0, s>>>(op->N, d, h, L.st, L.partials);
    BODY_CHECK();
  }
  cg32_update<<<rb, RED_THREADS, 0, s>>>(op->N, r, h, invd, L.st, L.partials, slots);
  BODY_CHECK();
  cg32_direction<<<rb, RED_THREADS, 0, s>>>(op->N, r, d, h, invd, x, 1, L.st, cond, use_cond, slots);
  BODY_CHECK();
  return FEPA_OK;
}

constexpr int STREAM_CHUNK = 8;

// Capture one iteration into the body of a while-node (once per loop and precond).
template <typename Body>
int build_while_graph(fepa_op* op, CgLoop& L, int precond, Body body) {
  TRY(prepare_f64(op));
  const int key = precond + 16 * (op->v32 + 1) + 256 * (op->v64 + 1) + 4096 * op->fuse_dot;
  if (L.exec && L.graph_key == key) return FEPA_OK;
  if (L.exec) { cudaGraphExecDestroy(L.exec); L.exec = nullptr; }
  if (L.graph) { cudaGraphDestroy(L.graph); L.graph = nullptr; }
  CUDA_TRY(cudaGraphCreate(&L.graph, 0));
  cudaGraphConditionalHandle cond;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, L.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CUDA_TRY(cudaGraphAddNode(&node, L.graph, nullptr, nullptr, 0, &np));
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  CUDA_TRY(cudaStreamBeginCaptureToGraph(op->cap_stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const int rc = body(op->cap_stream, cond, 1);
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(op->cap_stream, &captured);
  if (rc != FEPA_OK) return rc;
  if (ce != cudaSuccess) return fail(FEPA_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
  CUDA_TRY(cudaGraphInstantiate(&L.exec, L.graph, 0));
  L.graph_key = key;
  L.graph_kernels_per_iter = L.kernels_per_iter;  // set by the body just captured
  return FEPA_OK;
}

// Run iterations until the device sets done; leaves the final scalars in *out.
template <typename Body>
int run_loop(fepa_op* op, CgLoop& L, int precond, Body body, CgState* out) {
  cudaStream_t s = op->stream;
  TRY(prepare_f64(op));
  if (op->cg_mode == FEPA_CG_GRAPH) {
    TRY(build_while_graph(op, L, precond, body));
    CUDA_TRY(cudaGraphLaunch(L.exec, s));
    CUDA_TRY(cudaMemcpyAsync(out, L.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    g_launches.fetch_add(L.graph_kernels_per_iter * (int64_t)(out->iter > 0 ? out->iter : 1));
    return FEPA_OK;
  }
  for (;;) {
    for (int k = 0; k < STREAM_CHUNK; ++k) TRY(body(s, 0, 0));
    g_launches.fetch_add(L.kernels_per_iter * (int64_t)STREAM_CHUNK);
    CUDA_TRY(cudaMemcpyAsync(out, L.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (out->done) return FEPA_OK;
  }
}

// the loop stopped on a NaN or infinite ||r||^2 or ||b||^2 (non-finite input or breakdown)
bool nonfinite(const CgState& h) { return !std::isfinite(h.rr) || !std::isfinite(h.bb); }

int fail_nonfinite(const char* what) {
  return fail(FEPA_ERR_NONFINITE, "%s: a residual norm became NaN or infinite (non-finite b, x or operator data)",
              what);
}

void fill_stats(const CgState& h, fepa_cg_stats* stats) {
  if (!stats) return;
  stats->iterations = h.iter;
  stats->status = nonfinite(h) ? FEPA_ERR_NONFINITE : (h.converged ? FEPA_OK : FEPA_ERR_NOCONV);
  stats->b_norm = sqrt(h.bb);
  stats->rel_residual = h.bb > 0 ? sqrt(h.rr / h.bb) : 0.0;
  stats->precond_norm = sqrt(fabs(h.rho));
}

int check_solve_args(const fepa_op* op, const void* b, const void* x, double rtol, int maxit, int precond) {
  if (!op || !b || !x) return fail(FEPA_ERR_ARG, "null argument");
  if (maxit < 1) return fail(FEPA_ERR_ARG, "maxit must be >= 1");
  if (!(rtol >= 0.0)) return fail(FEPA_ERR_ARG, "rtol must be >= 0");
  if (precond != FEPA_PRECOND_NONE && precond != FEPA_PRECOND_JACOBI) return fail(FEPA_ERR_ARG, "bad precond");
  return FEPA_OK;
}

int run_cg(fepa_op* op, const double* b, double* x, double rtol, int maxit, int precond, fepa_cg_stats* stats) {
  TRY(check_solve_args(op, b, x, rtol, maxit, precond));
  CgLoop& L = op->cg64;
  TRY(ensure_loop<double>(op, L, false));
  if (!op->xw) TRY(dalloc(&op->xw, op->N));
  if (precond) TRY(ensure_inv_diag(op));
  const double* invd = precond ? op->inv_diag : nullptr;
  cudaStream_t s = op->stream;
  CUDA_TRY(cudaMemcpyAsync(op->xw, x, op->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemsetAsync(L.h, 0, op->N * sizeof(double), s));
  TRY(launch_apply(op, op->xw, (double*)L.h, nullptr, s));
  cg_init<<<L.red_blocks, RED_THREADS, 0, s>>>(op->N, b, (double*)L.r, (double*)L.d, (double*)L.h, invd, L.st,
                                                rtol * rtol, maxit, L.partials);
  LAUNCH_CHECK();
  auto body = [&](cudaStream_t bs, cudaGraphConditionalHandle cond, int use_cond) {
    return body64(op, L, invd, bs, cond, use_cond);
  };
  TRY(run_loop(op, L, precond, body, op->st_host));
  TRY(flush64(op, L, s));
  CUDA_TRY(cudaMemcpyAsync(x, op->xw, op->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const CgState h = *op->st_host;
  fill_stats(h, stats);
  if (nonfinite(h)) return fail_nonfinite("CG");
  if (!h.converged && rtol > 0.0)
    return fail(FEPA_ERR_NOCONV, "CG did not reach rtol %.3g in %d iterations (rel. residual %.3e)", rtol, h.iter,
                h.bb > 0 ? sqrt(h.rr / h.bb) : 0.0);
  return FEPA_OK;
}

// Mixed-precision solve: FP64 iterative refinement around an FP32 Jacobi-PCG (the inner
// tolerance of each step: inner_tol in cg_kernels.cuh).

// Power of two the FP64 residual of norm sqrt(rr) is scaled by before it enters the FP32 inner
// solve: 1 while its exponent is within +-20 (the common case: nothing to do), else the
// inverse of 2^exponent, so that FP32 products of the residual stay far from the float range's
// ends; the correction is scaled back exactly.
double residual_scale(double rr) {
  if (!(rr > 0.0) || !std::isfinite(rr)) return 1.0;
  const int k = ilogb(sqrt(rr));
  return (k > 20 || k < -20) ? ldexp(1.0, -k) : 1.0;
}

int run_refined(fepa_op* op, const double* b, double* x, double rtol, int max_outer, double inner_rtol,
                int inner_maxit, int precond, fepa_refine_stats* stats) {
  TRY(check_solve_args(op, b, x, rtol, max_outer, precond));
  if (!(inner_rtol > 0.0 && inner_rtol < 1.0)) return fail(FEPA_ERR_ARG, "inner_rtol must be in (0, 1)");
  if (inner_maxit < 1) return fail(FEPA_ERR_ARG, "inner_maxit must be >= 1");
  CgLoop& L = op->cg32;
  TRY(ensure_loop<float>(op, L, true));
  TRY(ensure_f32(op));
  if (!op->h64) {
    TRY(dalloc(&op->h64, op->N));
    TRY(dalloc(&op->st_ref, 1));
    TRY(dalloc(&op->partials_ref, 2 * (size_t)L.red_blocks));
    CUDA_TRY(cudaMemsetAsync(op->st_ref, 0, sizeof(CgState), op->stream));
  }
  cudaStream_t s = op->stream;
  if (precond) {
    TRY(ensure_inv_diag(op));
    if (!op->inv32_valid) {
      to_f32<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, op->inv_diag, (float*)L.invd);
      LAUNCH_CHECK();
      op->inv32_valid = true;
    }
  }
  const float* invd = precond ? (const float*)L.invd : nullptr;
  auto body = [&](cudaStream_t bs, cudaGraphConditionalHandle cond, int use_cond) {
    return body32(op, L, invd, bs, cond, use_cond);
  };
  int outer = 0, inner_total = 0;
  double rel = 0.0, bnorm = 0.0;
  CgState href;
  for (;;) {
    // FP64 residual r = b - A x
    CUDA_TRY(cudaMemsetAsync(op->h64, 0, op->N * sizeof(double), s));
    TRY(launch_apply(op, x, op->h64, nullptr, s));
    refine_residual<<<L.red_blocks, RED_THREADS, 0, s>>>(op->N, b, op->h64, (float*)L.r, op->st_ref,
                                                          op->partials_ref);
    LAUNCH_CHECK();
    CUDA_TRY(cudaMemcpyAsync(op->st_host, op->st_ref, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    href = *op->st_host;
    bnorm = sqrt(href.bb);
    rel = href.bb > 0 ? sqrt(href.rr / href.bb) : 0.0;
    if (!std::isfinite(href.rr) || !std::isfinite(href.bb)) rel = NAN;
    if (rel <= rtol || outer >= max_outer || std::isnan(rel)) break;
    // FP32 correction: A e = r with relative tolerance inner_rtol (relaxed on the last step)
    const double rs = residual_scale(href.rr);
    if (rs != 1.0) {
      refine_rescale<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, b, op->h64, (float*)L.r, rs);
      LAUNCH_CHECK();
    }
    const double tol = inner_tol(inner_rtol, rtol, rel);
    cg32_init<<<L.red_blocks, RED_THREADS, 0, s>>>(op->N, (const float*)L.r, (float*)L.x, (float*)L.r, (float*)L.d,
                                                    (float*)L.h, invd, L.st, tol * tol, inner_maxit, L.partials);
    LAUNCH_CHECK();
    CgState hin;
    TRY(run_loop(op, L, precond, body, &hin));
    inner_total += hin.iter;
    cg32_flush<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, (float*)L.x, (const float*)L.d, L.st);
    LAUNCH_CHECK();
    refine_correct<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, x, (const float*)L.x, 1.0 / rs);
    LAUNCH_CHECK();
    ++outer;
  }
  TRY(check_err(op));
  if (stats) {
    stats->outer_iterations = outer;
    stats->inner_iterations = inner_total;
    stats->rel_residual = rel;
    stats->b_norm = bnorm;
    stats->status = rel <= rtol ? FEPA_OK : (std::isnan(rel) ? FEPA_ERR_NONFINITE : FEPA_ERR_NOCONV);
  }
  if (std::isnan(rel)) return fail_nonfinite("refinement");
  if (rel > rtol)
    return fail(FEPA_ERR_NOCONV, "refinement did not reach rtol %.3g in %d outer steps (rel. residual %.3e)", rtol,
                outer, rel);
  return FEPA_OK;
}

// Mixed-precision CG with reliable updates (residual replacement): one FP32 Jacobi-PCG
// recurrence whose residual is replaced by the FP64 residual b - A x each time it has
// fallen by delta, the FP32 iterate being added to the FP64 x first.  Unlike the
// restarted refinement, the direction and the scalars carry over (cg32_replace), so the
// Krylov space is not thrown away at each correction.
int run_reliable(fepa_op* op, const double* b, double* x, double rtol, double delta, int maxit, int precond,
                 fepa_refine_stats* stats) {
  TRY(check_solve_args(op, b, x, rtol, maxit, precond));
  if (!(delta > 0.0 && delta < 1.0)) return fail(FEPA_ERR_ARG, "delta must be in (0, 1)");
  CgLoop& L = op->cg32;
  TRY(ensure_loop<float>(op, L, true));
  TRY(ensure_f32(op));
  if (!op->h64) {
    TRY(dalloc(&op->h64, op->N));
    TRY(dalloc(&op->st_ref, 1));
    TRY(dalloc(&op->partials_ref, 2 * (size_t)L.red_blocks));
    CUDA_TRY(cudaMemsetAsync(op->st_ref, 0, sizeof(CgState), op->stream));
  }
  cudaStream_t s = op->stream;
  if (precond) {
    TRY(ensure_inv_diag(op));
    if (!op->inv32_valid) {
      to_f32<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, op->inv_diag, (float*)L.invd);
      LAUNCH_CHECK();
      op->inv32_valid = true;
    }
  }
  const float* invd = precond ? (const float*)L.invd : nullptr;
  auto body = [&](cudaStream_t bs, cudaGraphConditionalHandle cond, int use_cond) {
    return body32(op, L, invd, bs, cond, use_cond);
  };
  double rs = 0.0;  // scale of the FP32 recurrence's units, fixed at the first residual
  auto residual = [&](double* rel, double* bb) -> int {  // FP64 r = b - A x into the FP32 loop's r
    CUDA_TRY(cudaMemsetAsync(op->h64, 0, op->N * sizeof(double), s));
    TRY(launch_apply(op, x, op->h64, nullptr, s));
    refine_residual<<<L.red_blocks, RED_THREADS, 0, s>>>(op->N, b, op->h64, (float*)L.r, op->st_ref,
                                                          op->partials_ref);
    LAUNCH_CHECK();
    CUDA_TRY(cudaMemcpyAsync(op->st_host, op->st_ref, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *bb = op->st_host->bb;
    *rel = op->st_host->bb > 0 ? sqrt(op->st_host->rr / op->st_host->bb) : 0.0;
    if (nonfinite(*op->st_host)) *rel = NAN;
    if (rs == 0.0) rs = residual_scale(op->st_host->rr);
    if (rs != 1.0) {
      refine_rescale<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, b, op->h64, (float*)L.r, rs);
      LAUNCH_CHECK();
    }
    return FEPA_OK;
  };
  double rel = 0.0, bb = 0.0;
  TRY(residual(&rel, &bb));
  const double rr0 = rel * rel * bb;
  const double floor2 = 0.25 * rtol * rtol * bb;  // a segment need not go below half the target
  int replacements = 0, iters = 0;
  if (rel > rtol) {  // (false for NaN: nothing to iterate on)
    const double first = rr0 > 0.0 && floor2 / rr0 > delta * delta ? floor2 / rr0 : delta * delta;
    cg32_init<<<L.red_blocks, RED_THREADS, 0, s>>>(op->N, (const float*)L.r, (float*)L.x, (float*)L.r, (float*)L.d,
                                                    (float*)L.h, invd, L.st, first, maxit, L.partials);
    LAUNCH_CHECK();
    for (;;) {
      CgState hin;
      TRY(run_loop(op, L, precond, body, &hin));
      iters = hin.iter;
      cg32_flush<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, (float*)L.x, (const float*)L.d, L.st);
      LAUNCH_CHECK();
      refine_correct<<<grid_for(op->N, 256, 148 * 16), 256, 0, s>>>(op->N, x, (const float*)L.x, 1.0 / rs);
      LAUNCH_CHECK();
      TRY(residual(&rel, &bb));
      if (rel <= rtol || iters >= maxit || std::isnan(rel)) break;
      cg32_replace<<<L.red_blocks, RED_THREADS, 0, s>>>(op->N, (const float*)L.r, (float*)L.x, invd, L.st,
                                                         delta * delta, floor2 * rs * rs, L.partials);
      LAUNCH_CHECK();
      cg32_direction<<<L.red_blocks, RED_THREADS, 0, s>>>(op->N, (const float*)L.r, (float*)L.d, (float*)L.h, invd,
                                                          nullptr, 0, L.st, 0, 0, nullptr);
      LAUNCH_CHECK();
      ++replacements;
    }
  }
  TRY(check_err(op));
  if (stats) {
    stats->outer_iterations = replacements;
    stats->inner_iterations = iters;
    stats->rel_residual = rel;
    stats->b_norm = sqrt(bb);
    stats->status = rel <= rtol ? FEPA_OK : (std::isnan(rel) ? FEPA_ERR_NONFINITE : FEPA_ERR_NOCONV);
  }
  if (std::isnan(rel)) return fail_nonfinite("reliable-update CG");
  if (rel > rtol)
    return fail(FEPA_ERR_NOCONV, "reliable-update CG did not reach rtol %.3g in %d iterations (rel. residual %.3e)",
                rtol, iters, rel);
  return FEPA_OK;
}

// host b/x: staged through op-owned device buffers
int host_solve(fepa_op* op, const double* b_host, double* x_host,
                      const std::function<int(const double*, double*)>& solve) {
  if (!op || !b_host || !x_host) return fail(FEPA_ERR_ARG, "null argument");
  if (!op->bw) TRY(dalloc(&op->bw, op->N));
  if (!op->xio) TRY(dalloc(&op->xio, op->N));
  cudaStream_t s = op->stream;
  CUDA_TRY(cudaMemcpyAsync(op->bw, b_host, op->N * sizeof(double), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(op->xio, x_host, op->N * sizeof(double), cudaMemcpyHostToDevice, s));
  int rc = solve(op->bw, op->xio);
  if (rc == FEPA_OK || rc == FEPA_ERR_NOCONV) {
    const std::string keep = g_err;
    cudaError_t e = cudaMemcpyAsync(x_host, op->xio, op->N * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(FEPA_ERR_CUDA, "host copy back: %s", cudaGetErrorString(e));
    g_err = keep;
  }
  return rc;
}

}  // namespace

extern "C" {

const char* fepa_version(void) { return "fepa 0.2 (sm_103a, FP64 and FP32 partial assembly)"; }

const char* fepa_last_error(void) { return g_err.c_str(); }

int64_t fepa_launch_count(void) { return g_launches.load(); }

}  // extern "C"

namespace {

// The part of op creation both mesh front ends share: checks of p, q and form, the 1D
// tables, device arrays, the vertex copy, G (written by build_map on the op's stream) and D.
// hex: the connectivity front end (conn_host and bdr_host already filled by the caller).
int create_common(fepa_op* op, int32_t p, int32_t q1d, int32_t form, void* stream, int64_t E, int64_t N,
                  int64_t nverts, const double* vertices, const std::function<int(fepa_op*)>& build_map) {
  if (p < 1 || p > FEPA_MAX_ORDER) return fail(FEPA_ERR_UNSUPPORTED, "order %d outside 1..%d", p, FEPA_MAX_ORDER);
  const int q = q1d == 0 ? p + 2 : q1d;
  if (q != p + 1 && q != p + 2) return fail(FEPA_ERR_UNSUPPORTED, "q1d %d not compiled for p=%d (p+1 or p+2)", q, p);
  if (form != FEPA_MASS && form != FEPA_DIFFUSION) return fail(FEPA_ERR_ARG, "unknown form %d", form);
  const int n = p + 1;
  if (N >= (int64_t)ESS_SKIP || E * n * n * n >= ((int64_t)1 << 31) || E >= ((int64_t)1 << 31))
    return fail(FEPA_ERR_ARG, "mesh too large for 32-bit DOF indices");
  op->p = p; op->q = q; op->n = n; op->form = form;
  op->E = E; op->N = N; op->nverts = nverts;
  op->stream = (cudaStream_t)stream;
  op->ks = kernels().t[p][q - p - 1][form];
  if (cudaGetDevice(&op->device) != cudaSuccess) return fail(FEPA_ERR_CUDA, "no CUDA device");
  if (cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(FEPA_ERR_CUDA, "stream creation failed");
  TRY(allow_smem((const void*)op->ks.apply, op->ks.apply_smem));
  for (int sh = 0; sh < 2; ++sh) TRY(allow_smem((const void*)op->ks.apply_df[sh], op->ks.df_smem[sh]));
  TRY(allow_smem((const void*)op->ks.diag_df, op->ks.diag_df_smem));
  TRY(allow_smem((const void*)op->ks.diag, op->ks.diag_smem));
  TRY(allow_smem((const void*)op->ks.rhs_df, op->ks.rhs_df_smem));

  // host tables
  std::vector<long double> nodes = basis::gll_nodes(p), gx, gw;
  basis::gauss_rule(q, gx, gw);
  std::vector<double> Bh, Gh;
  basis::lagrange_tables(nodes, gx, Bh, Gh);
  op->B32h.assign(Bh.begin(), Bh.end());
  op->G32h.assign(Gh.begin(), Gh.end());
  std::vector<double> ph(q), wh(q);
  for (int i = 0; i < q; ++i) { ph[i] = (double)gx[i]; wh[i] = (double)gw[i]; }

  const int ncomp = form == FEPA_DIFFUSION ? 6 : 1;
  const int64_t q3 = (int64_t)q * q * q;
  op->verts_host.assign(vertices, vertices + 3 * nverts);
  TRY(dalloc(&op->verts, 3 * nverts));
  TRY(dalloc(&op->gmap, E * n * n * n));
  TRY(dalloc(&op->qd, E * ncomp * q3));
  TRY(dalloc(&op->B, (size_t)q * n));
  TRY(dalloc(&op->G, (size_t)q * n));
  TRY(dalloc(&op->pts, q));
  TRY(dalloc(&op->wts, q));
  TRY(dalloc(&op->flag, 2));  // [0] mesh flags, [1] largest exponent of D
  TRY(dalloc(&op->err, 1));
  cudaStream_t s = op->stream;
  CUDA_TRY(cudaMemcpyAsync(op->verts, vertices, 3 * nverts * sizeof(double), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(op->B, Bh.data(), q * n * sizeof(double), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(op->G, Gh.data(), q * n * sizeof(double), cudaMemcpyHostToDevice, s));
  TRY(upload_df_tables(p, q, Bh, Gh, s));
  CUDA_TRY(cudaMemcpyAsync(op->pts, ph.data(), q * sizeof(double), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(op->wts, wh.data(), q * sizeof(double), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMallocHost((void**)&op->st_host_flag, 2 * sizeof(int)));
  CUDA_TRY(cudaMemsetAsync(op->flag, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(op->err, 0, sizeof(int), s));
  TRY(build_map(op));
  TRY(upload_gauss_df(q, gx, gw, s));
  TRY(compute_geometry(op));
  CUDA_TRY(cudaGetLastError());
  return read_mesh_flags(op);
}

}  // namespace

extern "C" {

int fepa_op_create(int32_t nx, int32_t ny, int32_t nz, const double* vertices, int32_t p, int32_t q1d, int32_t form,
                   void* stream, fepa_op** out) {
  if (!out) return fail(FEPA_ERR_ARG, "out is null");
  *out = nullptr;
  if (!vertices) return fail(FEPA_ERR_ARG, "vertices is null");
  if (nx < 1 || ny < 1 || nz < 1) return fail(FEPA_ERR_ARG, "element counts must be >= 1");
  const int64_t E = (int64_t)nx * ny * nz;
  const int64_t N = ((int64_t)p * nx + 1) * ((int64_t)p * ny + 1) * ((int64_t)p * nz + 1);
  const int64_t nv = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  fepa_op* op = new fepa_op();
  op->nx = nx; op->ny = ny; op->nz = nz;
  // G of the lexicographic node grid, built on the device
  auto grid_map = [](fepa_op* o) -> int {
    const int64_t slots = o->E * o->n * o->n * o->n;
    build_gmap<<<grid_for(slots, 256, 148 * 32), 256, 0, o->stream>>>(o->nx, o->ny, o->nz, o->p, 0, o->gmap);
    LAUNCH_CHECK();
    return FEPA_OK;
  };
  const int rc = create_common(op, p, q1d, form, stream, E, N, nv, vertices, grid_map);
  if (rc != FEPA_OK) { free_op(op); return rc; }
  *out = op;
  return FEPA_OK;
}

int fepa_hex_numbering(int64_t nverts, int64_t nelems, const int32_t* conn, int32_t p, int32_t* elem_dofs,
                       int64_t* ndofs) {
  if (!conn || !ndofs) return fail(FEPA_ERR_ARG, "null argument");
  if (p < 1 || p > FEPA_MAX_ORDER) return fail(FEPA_ERR_UNSUPPORTED, "order %d outside 1..%d", p, FEPA_MAX_ORDER);
  hexmesh::Numbering num;
  if (!hexmesh::number_dofs(nverts, nelems, conn, p, num, (int64_t)ESS_SKIP - 1))
    return fail(FEPA_ERR_MESH, "%s", num.error.c_str());
  *ndofs = num.ndofs;
  if (elem_dofs) std::copy(num.gmap.begin(), num.gmap.end(), elem_dofs);
  return FEPA_OK;
}

int fepa_op_create_hex(int64_t nverts, const double* vertices, int64_t nelems, const int32_t* conn, int32_t p,
                       int32_t q1d, int32_t form, void* stream, fepa_op** out) {
  if (!out) return fail(FEPA_ERR_ARG, "out is null");
  *out = nullptr;
  if (!vertices || !conn) return fail(FEPA_ERR_ARG, "null argument");
  if (nverts < 1 || nelems < 1 || nverts >= ((int64_t)1 << 31)) return fail(FEPA_ERR_ARG, "bad mesh sizes");
  if (p < 1 || p > FEPA_MAX_ORDER) return fail(FEPA_ERR_UNSUPPORTED, "order %d outside 1..%d", p, FEPA_MAX_ORDER);
  hexmesh::Numbering num;
  if (!hexmesh::number_dofs(nverts, nelems, conn, p, num, (int64_t)ESS_SKIP - 1))
    return fail(FEPA_ERR_MESH, "%s", num.error.c_str());
  fepa_op* op = new fepa_op();
  op->hex = true;
  op->nx = 1; op->ny = 1; op->nz = 1;
  op->conn_host.assign(conn, conn + 8 * nelems);
  op->bdr_host = std::move(num.boundary);
  const std::vector<int32_t>& gm = num.gmap;
  // G from the host numbering, and the connectivity the geometry kernels read
  auto copy_map = [&gm](fepa_op* o) -> int {
    TRY(dalloc(&o->econn, 8 * o->E));
    CUDA_TRY(cudaMemcpyAsync(o->econn, o->conn_host.data(), 8 * o->E * sizeof(int32_t), cudaMemcpyHostToDevice,
                             o->stream));
    CUDA_TRY(cudaMemcpyAsync(o->gmap, gm.data(), gm.size() * sizeof(int32_t), cudaMemcpyHostToDevice, o->stream));
    CUDA_TRY(cudaStreamSynchronize(o->stream));  // gm is a host temporary
    return FEPA_OK;
  };
  const int rc = create_common(op, p, q1d, form, stream, nelems, num.ndofs, nverts, vertices, copy_map);
  if (rc != FEPA_OK) { free_op(op); return rc; }
  *out = op;
  return FEPA_OK;
}

int fepa_op_set_vertices(fepa_op* op, const double* vertices, int32_t on_device) {
  if (!op || !vertices) return fail(FEPA_ERR_ARG, "null argument");
  cudaStream_t s = op->stream;
  const int64_t nv = op->nverts;
  CUDA_TRY(cudaMemcpyAsync(op->verts, vertices, 3 * nv * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (on_device) {
    op->verts_host.resize(3 * nv);
    CUDA_TRY(cudaMemcpyAsync(op->verts_host.data(), op->verts, 3 * nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  } else {
    op->verts_host.assign(vertices, vertices + 3 * nv);
  }
  CUDA_TRY(cudaMemsetAsync(op->flag, 0, sizeof(int), s));
  TRY(compute_geometry(op));  // refreshes D and its existing copies
  op->inv_diag_valid = false;
  op->inv32_valid = false;
  return read_mesh_flags(op);
}

void fepa_op_destroy(fepa_op* op) { free_op(op); }

int64_t fepa_op_ndofs(const fepa_op* op) { return op ? op->N : -1; }
int64_t fepa_op_nelems(const fepa_op* op) { return op ? op->E : -1; }
int32_t fepa_op_q1d(const fepa_op* op) { return op ? op->q : -1; }
int32_t fepa_op_dcomps(const fepa_op* op) { return op ? (op->form == FEPA_DIFFUSION ? 6 : 1) : -1; }

int fepa_op_set_stream(fepa_op* op, void* stream) {
  if (!op) return fail(FEPA_ERR_ARG, "op is null");
  op->stream = (cudaStream_t)stream;
  return FEPA_OK;
}

int fepa_test_set_first_wait_limit(int32_t iterations) {
  const int v = iterations < 0 ? WAIT_LIMIT : iterations;
  CUDA_TRY(cudaMemcpyToSymbol(c_first_wait_limit, &v, sizeof(int)));
  CUDA_TRY(cudaDeviceSynchronize());
  return FEPA_OK;
}

int fepa_op_set_fused_dot(fepa_op* op, int32_t enable) {
  if (!op) return fail(FEPA_ERR_ARG, "op is null");
  op->fuse_dot = enable ? 1 : 0;
  return FEPA_OK;
}

int fepa_op_set_cg_mode(fepa_op* op, int32_t mode) {
  if (!op) return fail(FEPA_ERR_ARG, "op is null");
  if (mode != FEPA_CG_GRAPH && mode != FEPA_CG_STREAM) return fail(FEPA_ERR_ARG, "unknown CG mode %d", mode);
  op->cg_mode = mode;
  return FEPA_OK;
}

int fepa_op_boundary_dofs(const fepa_op* op, int32_t* dofs, int64_t capacity, int64_t* count) {
  if (!op || !count) return fail(FEPA_ERR_ARG, "null argument");
  if (op->hex) {
    const int64_t total = (int64_t)op->bdr_host.size();
    *count = total;
    if (!dofs) return FEPA_OK;
    if (capacity < total)
      return fail(FEPA_ERR_ARG, "capacity %lld < %lld boundary DOFs", (long long)capacity, (long long)total);
    std::copy(op->bdr_host.begin(), op->bdr_host.end(), dofs);
    return FEPA_OK;
  }
  const int64_t Nx = (int64_t)op->p * op->nx + 1, Ny = (int64_t)op->p * op->ny + 1, Nz = (int64_t)op->p * op->nz + 1;
  const int64_t total = Nx * Ny * Nz - (Nx - 2) * (Ny - 2) * (Nz - 2);
  *count = total;
  if (!dofs) return FEPA_OK;
  if (capacity < total) return fail(FEPA_ERR_ARG, "capacity %lld < %lld boundary DOFs", (long long)capacity, (long long)total);
  int64_t k = 0;
  for (int64_t z = 0; z < Nz; ++z)
    for (int64_t y = 0; y < Ny; ++y)
      for (int64_t x = 0; x < Nx; ++x)
        if (x == 0 || y == 0 || z == 0 || x == Nx - 1 || y == Ny - 1 || z == Nz - 1)
          dofs[k++] = (int32_t)(x + Nx * (y + Ny * z));
  return FEPA_OK;
}

int fepa_op_set_essential(fepa_op* op, const int32_t* dofs, int64_t count) {
  if (!op) return fail(FEPA_ERR_ARG, "op is null");
  if (count < 0 || (count > 0 && !dofs)) return fail(FEPA_ERR_ARG, "bad essential list");
  for (int64_t i = 0; i < count; ++i)
    if (dofs[i] < 0 || dofs[i] >= op->N) return fail(FEPA_ERR_ARG, "essential DOF %d out of range", dofs[i]);
  cudaStream_t s = op->stream;
  std::vector<unsigned char> mask(op->N, 0);
  for (int64_t i = 0; i < count; ++i) mask[dofs[i]] = 1;
  unsigned char* dmask = nullptr;
  TRY(dalloc(&dmask, op->N));
  cudaError_t e = cudaMemcpyAsync(dmask, mask.data(), op->N, cudaMemcpyHostToDevice, s);
  int* first = nullptr;  // unstructured mesh: first slot of every DOF, its owner when essential
  if (e == cudaSuccess && op->hex) {
    if (dalloc(&first, op->N) != FEPA_OK) {
      cudaFree(dmask);
      return FEPA_ERR_OOM;
    }
    e = cudaMemsetAsync(first, 0x7f, op->N * sizeof(int), s);
  }
  if (e == cudaSuccess) {
    const int64_t total = op->E * op->n * op->n * op->n;
    const int grid = grid_for(total, 256, 148 * 32);
    if (op->hex) {
      gmap_first_slot<<<grid, 256, 0, s>>>(total, op->gmap, first);
      flag_gmap_first<<<grid, 256, 0, s>>>(total, dmask, first, op->gmap);
      g_launches.fetch_add(2);
    } else {
      flag_gmap<<<grid, 256, 0, s>>>(op->nx, op->ny, op->nz, op->p, dmask, op->gmap);
      g_launches.fetch_add(1);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dmask);
  if (first) cudaFree(first);
  if (e != cudaSuccess) return fail(FEPA_ERR_CUDA, "set_essential: %s", cudaGetErrorString(e));
  if (op->ess) { cudaFree(op->ess); op->ess = nullptr; }
  op->ess_count = 0;
  if (count > 0) {
    TRY(dalloc(&op->ess, count));
    CUDA_TRY(cudaMemcpy(op->ess, dofs, count * sizeof(int32_t), cudaMemcpyHostToDevice));
    op->ess_count = count;
  }
  op->inv_diag_valid = false;
  op->inv32_valid = false;
  return FEPA_OK;
}

int fepa_op_elem_dofs(const fepa_op* op, int32_t* out) {
  if (!op || !out) return fail(FEPA_ERR_ARG, "null argument");
  const int64_t total = op->E * op->n * op->n * op->n;
  unflag_gmap<<<grid_for(total, 256, 148 * 32), 256, 0, op->stream>>>(total, op->gmap, out);
  LAUNCH_CHECK();
  return FEPA_OK;
}

int fepa_op_qdata(const fepa_op* op, double* out) {
  if (!op || !out) return fail(FEPA_ERR_ARG, "null argument");
  const int64_t count = op->E * (op->form == FEPA_DIFFUSION ? 6 : 1) * (int64_t)op->q * op->q * op->q;
  CUDA_TRY(cudaMemcpyAsync(out, op->qd, count * sizeof(double), cudaMemcpyDeviceToDevice, op->stream));
  return FEPA_OK;
}

int fepa_op_qp_coords(const fepa_op* op, double* out) {
  if (!op || !out) return fail(FEPA_ERR_ARG, "null argument");
  const int64_t total = op->E * op->q * op->q * op->q;
  qp_coords_kernel<<<grid_for(total, 256, 148 * 32), 256, 0, op->stream>>>(op->E, op->nx, op->ny, op->econn, op->q,
                                                                         op->verts, op->pts, out);
  LAUNCH_CHECK();
  return FEPA_OK;
}

int fepa_op_apply(fepa_op* op, const double* x, double* y) {
  if (!op || !x || !y) return fail(FEPA_ERR_ARG, "null argument");
  if (x == y) return fail(FEPA_ERR_ARG, "x and y must not alias");
  CUDA_TRY(cudaMemsetAsync(y, 0, op->N * sizeof(double), op->stream));
  return launch_apply(op, x, y, nullptr, op->stream);
}

int fepa_op_apply_f32(fepa_op* op, const float* x, float* y) {
  if (!op || !x || !y) return fail(FEPA_ERR_ARG, "null argument");
  if (x == y) return fail(FEPA_ERR_ARG, "x and y must not alias");
  TRY(ensure_f32(op));
  CUDA_TRY(cudaMemsetAsync(y, 0, op->N * sizeof(float), op->stream));
  TRY(launch_apply32_nocount(op, x, y, nullptr, op->stream));
  g_launches.fetch_add(1);
  return FEPA_OK;
}

int fepa_op_apply_f32_dot(fepa_op* op, const float* x, float* y, double* xax) {
  if (!op || !x || !y || !xax) return fail(FEPA_ERR_ARG, "null argument");
  if (x == y) return fail(FEPA_ERR_ARG, "x and y must not alias");
  TRY(ensure_f32(op));
  cudaStream_t s = op->stream;
  if (!op->dot_slots) {
    TRY(dalloc(&op->dot_slots, DOT_SLOTS));
    CUDA_TRY(cudaMemsetAsync(op->dot_slots, 0, DOT_SLOTS * sizeof(double), s));
  }
  CUDA_TRY(cudaMemsetAsync(y, 0, op->N * sizeof(float), s));
  if (has_dot_build(op, op->v32)) {
    TRY(launch_apply32_variant(op, op->v32, x, y, nullptr, s, op->dot_slots));
    g_launches.fetch_add(1);
  } else {
    TRY(launch_apply32_variant(op, op->v32, x, y, nullptr, s));
    dot32_slots<<<grid_for(op->N, RED_THREADS, 148 * 8), RED_THREADS, 0, s>>>(op->N, x, y, op->dot_slots);
    LAUNCH_CHECK();
    g_launches.fetch_add(2);
  }
  dot_collect<<<1, RED_THREADS, 0, s>>>(op->dot_slots, xax);
  LAUNCH_CHECK();
  g_launches.fetch_add(1);
  return FEPA_OK;
}

int fepa_op_set_f32_variant(fepa_op* op, int32_t variant) {
  if (!op) return fail(FEPA_ERR_ARG, "op is null");
  if (variant < -1 || variant >= N32_VARIANTS) return fail(FEPA_ERR_ARG, "variant %d outside -1..%d", variant,
                                                            N32_VARIANTS - 1);
  op->v32_forced = variant;
  op->v32 = variant;  // -1: choose again at next use
  return FEPA_OK;
}

int32_t fepa_op_f32_variant(const fepa_op* op) { return op ? op->v32 : -1; }

int fepa_op_set_f64_variant(fepa_op* op, int32_t variant) {
  if (!op) return fail(FEPA_ERR_ARG, "op is null");
  if (variant < -1 || variant >= N64_VARIANTS) return fail(FEPA_ERR_ARG, "variant %d outside -1..%d", variant,
                                                            N64_VARIANTS - 1);
  op->v64_forced = variant;
  op->v64 = variant;  // -1: choose again at next use
  return FEPA_OK;
}

int32_t fepa_op_f64_variant(const fepa_op* op) { return op ? op->v64 : -1; }

const char* fepa_f64_variant_name(int32_t variant) {
  static const char* names[N64_VARIANTS] = {"FP64 pipe (DFMA)", "double-float on the FP32 pipe",
                                             "double-float on the FP32 pipe, half block"};
  return (variant >= 0 && variant < N64_VARIANTS) ? names[variant] : "unknown";
}

const char* fepa_f32_variant_name(int32_t variant) {
  static const char* names[N32_VARIANTS] = {"tma-staged D", "direct D", "direct D, half block",
                                             "persistent pipeline (TMA D, cp.async gather)"};
  return (variant >= 0 && variant < N32_VARIANTS) ? names[variant] : "unknown";
}

int fepa_op_diagonal(fepa_op* op, double* diag) {
  if (!op || !diag) return fail(FEPA_ERR_ARG, "null argument");
  return compute_diagonal(op, diag, op->stream);
}

// load vector in double-float (FP64-accurate; the FP64 pipe would spend ~90 % of the time
// on the three FP64 sines per point)
static int rhs_common(fepa_op* op, const double* f_qp, double scale, double* b) {
  cudaStream_t s = op->stream;
  CUDA_TRY(cudaMemsetAsync(b, 0, op->N * sizeof(double), s));
  const KernelSet& k = op->ks;
  const int grid = (int)((op->E + k.rhs_df_ne - 1) / k.rhs_df_ne);
  // the sine's amplitude enters as m 2^k (m in [0.5, 1)): m in the kernel, 2^k on the FP64 result, so any
  // FP64 amplitude keeps the double-float products in range
  int k2 = 0;
  const double m = !f_qp && scale != 0.0 && std::isfinite(scale) ? frexp(scale, &k2) : scale;
  k.rhs_df<<<grid, dim3(op->q * op->q, k.rhs_df_ne), k.rhs_df_smem, s>>>(op->E, op->nx, op->ny, op->econn,
                                                                         op->verts_df, op->gmap, f_qp, m,
                                                                         ldexp(1.0, k2), b);
  LAUNCH_CHECK();
  return FEPA_OK;
}

int fepa_op_rhs(fepa_op* op, const double* f_qp, double* b) {
  if (!op || !f_qp || !b) return fail(FEPA_ERR_ARG, "null argument");
  return rhs_common(op, f_qp, 1.0, b);
}

int fepa_op_rhs_sine(fepa_op* op, double scale, double* b) {
  if (!op || !b) return fail(FEPA_ERR_ARG, "null argument");
  TRY(rhs_common(op, nullptr, scale, b));
  if (op->ess_count > 0) {
    set_rows<<<grid_for(op->ess_count, 256, 148 * 8), 256, 0, op->stream>>>(op->ess_count, op->ess, 0.0, b);
    LAUNCH_CHECK();
  }
  return FEPA_OK;
}

int fepa_cg_solve(fepa_op* op, const double* b, double* x, double rtol, int32_t maxit, int32_t precond,
                  fepa_cg_stats* stats) {
  return run_cg(op, b, x, rtol, maxit, precond, stats);
}

int fepa_cg_solve_host(fepa_op* op, const double* b_host, double* x_host, double rtol, int32_t maxit, int32_t precond,
                       fepa_cg_stats* stats) {
  return host_solve(op, b_host, x_host, [&](const double* b, double* x) {
    return run_cg(op, b, x, rtol, maxit, precond, stats);
  });
}

int fepa_cg_iterations(fepa_op* op, const double* b, double* x, int32_t iters, int32_t precond, fepa_cg_stats* stats) {
  if (iters < 1) return fail(FEPA_ERR_ARG, "iters must be >= 1");
  return run_cg(op, b, x, 0.0, iters, precond, stats);
}

int fepa_solve_refined(fepa_op* op, const double* b, double* x, double rtol, int32_t max_outer, double inner_rtol,
                       int32_t inner_maxit, int32_t precond, fepa_refine_stats* stats) {
  return run_refined(op, b, x, rtol, max_outer, inner_rtol, inner_maxit, precond, stats);
}

int fepa_solve_reliable(fepa_op* op, const double* b, double* x, double rtol, double delta, int32_t maxit,
                        int32_t precond, fepa_refine_stats* stats) {
  return run_reliable(op, b, x, rtol, delta, maxit, precond, stats);
}

int fepa_solve_reliable_host(fepa_op* op, const double* b_host, double* x_host, double rtol, double delta,
                             int32_t maxit, int32_t precond, fepa_refine_stats* stats) {
  return host_solve(op, b_host, x_host, [&](const double* b, double* x) {
    return run_reliable(op, b, x, rtol, delta, maxit, precond, stats);
  });
}

int fepa_solve_refined_host(fepa_op* op, const double* b_host, double* x_host, double rtol, int32_t max_outer,
                            double inner_rtol, int32_t inner_maxit, int32_t precond, fepa_refine_stats* stats) {
  return host_solve(op, b_host, x_host, [&](const double* b, double* x) {
    return run_refined(op, b, x, rtol, max_outer, inner_rtol, inner_maxit, precond, stats);
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// CG solve without allocation (fepa_cg_solve_noalloc).  Its work vectors live in
// one file-scope device array instead of cudaMalloc'ed buffers, for callers that
// cannot allocate device memory after start-up.  Layout, in doubles, each piece
// starting on a 256-byte boundary:
//   [0, 32)                     CgState (device scalars and the reduction ticket)
//   [32, 32 + 3584)             block partial sums of the dot products
//   then r, d, h, 1/diag        FEPA_NOALLOC_MAX_DOFS doubles each
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NA_STATE = 0;
constexpr int64_t NA_PARTIALS = 32;
constexpr int64_t NA_PARTIALS_CAP = 3584;  // >= 3 * (148 * 8) block partials
constexpr int64_t NA_VEC0 = NA_PARTIALS + NA_PARTIALS_CAP;
constexpr int64_t NA_TOTAL = NA_VEC0 + 4 * (int64_t)FEPA_NOALLOC_MAX_DOFS;
static_assert(sizeof(CgState) <= 32 * sizeof(double), "state does not fit its slot");
static_assert(NA_VEC0 % 32 == 0 && FEPA_NOALLOC_MAX_DOFS % 32 == 0, "pieces must stay 256-byte aligned");

static __device__ __align__(256) double g_noalloc_scratch[NA_TOTAL];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[NA_MAX_DEVICES] = {nullptr};

// Device address of the array on the current device, looked up once per device.
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= NA_MAX_DEVICES) return fail(FEPA_ERR_ARG, "device ordinal %d unsupported", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    int cur = -1;
    CUDA_TRY(cudaGetDevice(&cur));
    if (cur != device) return fail(FEPA_ERR_ARG, "the op's device %d is not the current device %d", device, cur);
    void* p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[device] = (double*)p;
  }
  *out = g_noalloc_ptr[device];
  return FEPA_OK;
}

}  // namespace

extern "C" int fepa_cg_solve_noalloc(fepa_op* op, const double* b, double* x, double rtol, int32_t maxit,
                                     int32_t precond, fepa_cg_stats* stats) {
  if (!op || !b || !x) return fail(FEPA_ERR_ARG, "null argument");
  if (maxit < 1) return fail(FEPA_ERR_ARG, "maxit must be >= 1");
  if (!(rtol >= 0.0)) return fail(FEPA_ERR_ARG, "rtol must be >= 0");
  if (precond != FEPA_PRECOND_NONE && precond != FEPA_PRECOND_JACOBI) return fail(FEPA_ERR_ARG, "bad precond");
  if (op->N > FEPA_NOALLOC_MAX_DOFS)
    return fail(FEPA_ERR_ARG, "fepa_cg_solve_noalloc handles at most %d DOFs; this operator has %lld",
                FEPA_NOALLOC_MAX_DOFS, (long long)op->N);
  double* base = nullptr;
  TRY(noalloc_scratch(op->device, &base));
  CgState* st = (CgState*)(base + NA_STATE);
  double* partials = base + NA_PARTIALS;
  double* r = base + NA_VEC0;
  double* d = r + FEPA_NOALLOC_MAX_DOFS;
  double* h = d + FEPA_NOALLOC_MAX_DOFS;
  double* invd = h + FEPA_NOALLOC_MAX_DOFS;
  const int64_t N = op->N;
  const int rb = grid_for(N, RED_THREADS, 148 * 8);
  cudaStream_t s = op->stream;

  // the array holds whatever the previous call left: reset the scalars and ticket
  CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(CgState), s));
  if (precond) {
    TRY(compute_diagonal(op, invd, s, false));  // zeroes invd, then sums the element diagonals
    reciprocal<<<grid_for(N, 256, 148 * 16), 256, 0, s>>>(N, invd, invd);
    LAUNCH_CHECK();
  }
  const double* pinv = precond ? invd : nullptr;
  CUDA_TRY(cudaMemsetAsync(h, 0, N * sizeof(double), s));
  TRY(launch_apply_untuned(op, x, h, nullptr, s));
  cg_init<<<rb, RED_THREADS, 0, s>>>(N, b, r, d, h, pinv, st, rtol * rtol, maxit, partials);
  LAUNCH_CHECK();
  // host-driven loop in chunks; every kernel returns at once after the device sets done
  constexpr int CHUNK = 8;
  CgState hs;
  for (;;) {
    for (int k = 0; k < CHUNK; ++k) {
      TRY(launch_apply_untuned(op, d, h, &st->done, s));
      cg_dot_dh<<<rb, RED_THREADS, 0, s>>>(N, d, h, st, partials);
      LAUNCH_CHECK();
      cg_update<<<rb, RED_THREADS, 0, s>>>(N, x, r, d, h, pinv, st, partials);
      LAUNCH_CHECK();
      cg_direction<<<rb, RED_THREADS, 0, s>>>(N, r, d, h, pinv, st, 0, 0);
      LAUNCH_CHECK();
    }
    CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.done) break;
  }
  if (stats) {
    stats->iterations = hs.iter;
    stats->status = nonfinite(hs) ? FEPA_ERR_NONFINITE : (hs.converged ? FEPA_OK : FEPA_ERR_NOCONV);
    stats->b_norm = sqrt(hs.bb);
    stats->rel_residual = hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0;
    stats->precond_norm = sqrt(fabs(hs.rho));
  }
  if (nonfinite(hs)) return fail_nonfinite("CG");
  if (!hs.converged && rtol > 0.0)
    return fail(FEPA_ERR_NOCONV, "CG did not reach rtol %.3g in %d iterations (rel. residual %.3e)", rtol, hs.iter,
                hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0);
  return FEPA_OK;
}

#include "batch_api.inc"
#include "solver_api.inc"
#include "mg_api.inc"
