// C-ABI of the partial-assembly library (declarations and conventions: include/fepa.h).
//
// Host side: validates arguments, builds the 1D tables, owns device arrays, dispatches
// the compiled (p, q, form) kernel instances, and drives CG through a CUDA graph whose
// while-node repeats one CG iteration until a device-side flag says stop.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fepa.h"
#include "basis1d.hpp"
#include "cg_kernels.cuh"
#include "pa_kernels.cuh"

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

#define LAUNCH_CHECK()                                                                               \
  do {                                                                                               \
    g_launches.fetch_add(1);                                                                         \
    cudaError_t e_ = cudaGetLastError();                                                             \
    if (e_ != cudaSuccess) return fail(FEPA_ERR_CUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                          \
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
struct KernelSet {
  void (*apply)(int, const int*, const double*, const double*, const double*, const double*, double*, const int*);
  void (*diag)(int, const int*, const double*, const double*, const double*, double*);
  void (*rhs)(int, int, const double*, const int*, const double*, const double*, const double*, const double*,
              double, double*);
  int apply_smem, apply_tpe, apply_ne;
  int diag_smem, rhs_smem;
};

template <int P, int Q, bool DIFF>
KernelSet make_set() {
  KernelSet k;
  k.apply = pa_apply_f64<P, Q, DIFF>;
  k.diag = pa_diag_f64<P, Q, DIFF>;
  k.rhs = pa_rhs_f64<P, Q>;
  k.apply_smem = PaShape<P, Q, DIFF>::SMEM;
  k.apply_tpe = PaShape<P, Q, DIFF>::TPE;
  k.apply_ne = PaShape<P, Q, DIFF>::NE;
  k.diag_smem = DiagShape<P, Q, DIFF>::SMEM;
  k.rhs_smem = RhsShape<P, Q>::SMEM;
  return k;
}

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

int allow_smem(const void* fn, int bytes) {
  if (bytes > 48 * 1024) CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return FEPA_OK;
}

}  // namespace

struct fepa_op {
  int nx, ny, nz, p, q, n, form;
  int64_t E, N;
  int device;
  cudaStream_t stream;
  cudaStream_t cap_stream;  // private stream used only to capture graphs
  KernelSet ks;
  // device arrays owned by the op
  double* verts = nullptr;
  int* gmap = nullptr;
  double* qd = nullptr;
  double* B = nullptr;
  double* G = nullptr;
  double* pts = nullptr;
  double* wts = nullptr;
  int* ess = nullptr;
  int64_t ess_count = 0;
  int* flag = nullptr;  // device int used for mesh checks
  // CG workspace (allocated on first solve)
  double* inv_diag = nullptr;
  bool inv_diag_valid = false;
  double *r = nullptr, *d = nullptr, *h = nullptr, *xw = nullptr, *bw = nullptr, *xio = nullptr;
  CgState* st = nullptr;
  double* partials = nullptr;
  int red_blocks = 0;
  CgState* st_host = nullptr;  // pinned
  int* st_host_flag = nullptr;  // pinned
  cudaGraphExec_t graph_exec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_precond = -1;
};

namespace {

void free_op(fepa_op* op) {
  if (!op) return;
  cudaStreamSynchronize(op->stream);
  if (op->graph_exec) cudaGraphExecDestroy(op->graph_exec);
  if (op->graph) cudaGraphDestroy(op->graph);
  for (void* p : {(void*)op->verts, (void*)op->gmap, (void*)op->qd, (void*)op->B, (void*)op->G, (void*)op->pts,
                  (void*)op->wts, (void*)op->ess, (void*)op->flag, (void*)op->inv_diag, (void*)op->r, (void*)op->d,
                  (void*)op->h, (void*)op->xw, (void*)op->bw, (void*)op->xio, (void*)op->st, (void*)op->partials})
    if (p) cudaFree(p);
  if (op->st_host) cudaFreeHost(op->st_host);
  if (op->st_host_flag) cudaFreeHost(op->st_host_flag);
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

#define TRY(call)              \
  do {                         \
    int rc_ = (call);          \
    if (rc_ != FEPA_OK) return rc_; \
  } while (0)

int launch_apply(fepa_op* op, const double* x, double* y, const int* skip, cudaStream_t s) {
  const KernelSet& k = op->ks;
  const int grid = (int)((op->E + k.apply_ne - 1) / k.apply_ne);
  k.apply<<<grid, dim3(k.apply_tpe, k.apply_ne), k.apply_smem, s>>>((int)op->E, op->gmap, op->qd, op->B, op->G, x, y,
                                                                    skip);
  LAUNCH_CHECK();
  return FEPA_OK;
}

int ensure_workspace(fepa_op* op) {
  if (op->r) return FEPA_OK;
  TRY(dalloc(&op->r, op->N));
  TRY(dalloc(&op->d, op->N));
  TRY(dalloc(&op->h, op->N));
  TRY(dalloc(&op->xw, op->N));
  TRY(dalloc(&op->st, 1));
  op->red_blocks = grid_for(op->N, RED_THREADS, 148 * 8);
  TRY(dalloc(&op->partials, 3 * (size_t)op->red_blocks));
  CUDA_TRY(cudaMemsetAsync(op->st, 0, sizeof(CgState), op->stream));
  CUDA_TRY(cudaMallocHost((void**)&op->st_host, sizeof(CgState)));
  return FEPA_OK;
}

int compute_diagonal(fepa_op* op, double* out, cudaStream_t s) {
  CUDA_TRY(cudaMemsetAsync(out, 0, op->N * sizeof(double), s));
  op->ks.diag<<<(int)op->E, op->q * op->q, op->ks.diag_smem, s>>>((int)op->E, op->gmap, op->qd, op->B, op->G, out);
  LAUNCH_CHECK();
  return FEPA_OK;
}

int ensure_inv_diag(fepa_op* op) {
  if (op->inv_diag_valid) return FEPA_OK;
  if (!op->inv_diag) TRY(dalloc(&op->inv_diag, op->N));
  TRY(compute_diagonal(op, op->inv_diag, op->stream));
  reciprocal<<<grid_for(op->N, 256, 148 * 16), 256, 0, op->stream>>>(op->N, op->inv_diag, op->inv_diag);
  LAUNCH_CHECK();
  op->inv_diag_valid = true;
  return FEPA_OK;
}

// One CG iteration as four kernels, captured into the body of a while-node.
int build_graph(fepa_op* op, int precond) {
  if (op->graph_exec && op->graph_precond == precond) return FEPA_OK;
  if (op->graph_exec) {
    cudaGraphExecDestroy(op->graph_exec);
    op->graph_exec = nullptr;
  }
  if (op->graph) {
    cudaGraphDestroy(op->graph);
    op->graph = nullptr;
  }
  CUDA_TRY(cudaGraphCreate(&op->graph, 0));
  cudaGraphConditionalHandle cond;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, op->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CUDA_TRY(cudaGraphAddNode(&node, op->graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CUDA_TRY(cudaStreamBeginCaptureToGraph(op->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const double* invd = precond ? op->inv_diag : nullptr;
  const int rb = op->red_blocks;
  int rc = launch_apply(op, op->d, op->h, &op->st->done, op->cap_stream);
  if (rc == FEPA_OK) {
    cg_dot_dh<<<rb, RED_THREADS, 0, op->cap_stream>>>(op->N, op->d, op->h, op->st, op->partials);
    cg_update<<<rb, RED_THREADS, 0, op->cap_stream>>>(op->N, op->xw, op->r, op->d, op->h, invd, op->st, op->partials);
    cg_direction<<<rb, RED_THREADS, 0, op->cap_stream>>>(op->N, op->r, op->d, op->h, invd, op->st, cond, 1);
  }
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(op->cap_stream, &captured);
  g_launches.fetch_sub(1);  // the captured apply did not run
  if (rc != FEPA_OK) return rc;
  if (ce != cudaSuccess) return fail(FEPA_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaGraphInstantiate(&op->graph_exec, op->graph, 0));
  op->graph_precond = precond;
  return FEPA_OK;
}

int run_cg(fepa_op* op, const double* b, double* x, double rtol, int maxit, int precond, fepa_cg_stats* stats) {
  if (!op || !b || !x) return fail(FEPA_ERR_ARG, "null argument");
  if (maxit < 1) return fail(FEPA_ERR_ARG, "maxit must be >= 1");
  if (!(rtol >= 0.0)) return fail(FEPA_ERR_ARG, "rtol must be >= 0");
  if (precond != FEPA_PRECOND_NONE && precond != FEPA_PRECOND_JACOBI) return fail(FEPA_ERR_ARG, "bad precond");
  TRY(ensure_workspace(op));
  if (precond) TRY(ensure_inv_diag(op));
  TRY(build_graph(op, precond));
  cudaStream_t s = op->stream;
  const int rb = op->red_blocks;
  CUDA_TRY(cudaMemcpyAsync(op->xw, x, op->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemsetAsync(op->h, 0, op->N * sizeof(double), s));
  TRY(launch_apply(op, op->xw, op->h, nullptr, s));
  cg_init<<<rb, RED_THREADS, 0, s>>>(op->N, b, op->r, op->d, op->h, precond ? op->inv_diag : nullptr, op->st,
                                      rtol * rtol, maxit, op->partials);
  LAUNCH_CHECK();
  CUDA_TRY(cudaGraphLaunch(op->graph_exec, s));
  CUDA_TRY(cudaMemcpyAsync(x, op->xw, op->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(op->st_host, op->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const CgState& h = *op->st_host;
  g_launches.fetch_add(4 * (int64_t)(h.iter > 0 ? h.iter : 1));
  if (stats) {
    stats->iterations = h.iter;
    stats->status = h.converged ? FEPA_OK : FEPA_ERR_NOCONV;
    stats->b_norm = sqrt(h.bb);
    stats->rel_residual = h.bb > 0 ? sqrt(h.rr / h.bb) : 0.0;
    stats->precond_norm = sqrt(fabs(h.rho));
  }
  if (!h.converged && rtol > 0.0)
    return fail(FEPA_ERR_NOCONV, "CG did not reach rtol %.3g in %d iterations (rel. residual %.3e)", rtol, h.iter,
                h.bb > 0 ? sqrt(h.rr / h.bb) : 0.0);
  return FEPA_OK;
}

}  // namespace

extern "C" {

const char* fepa_version(void) { return "fepa 0.1 (sm_103a, FP64 partial assembly)"; }

const char* fepa_last_error(void) { return g_err.c_str(); }

int64_t fepa_launch_count(void) { return g_launches.load(); }

int fepa_op_create(int32_t nx, int32_t ny, int32_t nz, const double* vertices, int32_t p, int32_t q1d, int32_t form,
                   void* stream, fepa_op** out) {
  if (!out) return fail(FEPA_ERR_ARG, "out is null");
  *out = nullptr;
  if (!vertices) return fail(FEPA_ERR_ARG, "vertices is null");
  if (nx < 1 || ny < 1 || nz < 1) return fail(FEPA_ERR_ARG, "element counts must be >= 1");
  if (p < 1 || p > FEPA_MAX_ORDER) return fail(FEPA_ERR_UNSUPPORTED, "order %d outside 1..%d", p, FEPA_MAX_ORDER);
  const int q = q1d == 0 ? p + 2 : q1d;
  if (q != p + 1 && q != p + 2) return fail(FEPA_ERR_UNSUPPORTED, "q1d %d not compiled for p=%d (p+1 or p+2)", q, p);
  if (form != FEPA_MASS && form != FEPA_DIFFUSION) return fail(FEPA_ERR_ARG, "unknown form %d", form);
  const int64_t E = (int64_t)nx * ny * nz;
  const int n = p + 1;
  const int64_t N = ((int64_t)p * nx + 1) * ((int64_t)p * ny + 1) * ((int64_t)p * nz + 1);
  if (N >= (int64_t)ESS_SKIP || E * n * n * n >= ((int64_t)1 << 31) || E >= ((int64_t)1 << 31))
    return fail(FEPA_ERR_ARG, "mesh too large for 32-bit DOF indices");

  fepa_op* op = new fepa_op();
  op->nx = nx; op->ny = ny; op->nz = nz; op->p = p; op->q = q; op->n = n; op->form = form;
  op->E = E; op->N = N;
  op->stream = (cudaStream_t)stream;
  op->ks = kernels().t[p][q - p - 1][form];
  auto bail = [&](int rc) { free_op(op); return rc; };
  if (cudaGetDevice(&op->device) != cudaSuccess) return bail(fail(FEPA_ERR_CUDA, "no CUDA device"));
  if (cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(FEPA_ERR_CUDA, "stream creation failed"));
  int rc;
  if ((rc = allow_smem((const void*)op->ks.apply, op->ks.apply_smem)) ||
      (rc = allow_smem((const void*)op->ks.diag, op->ks.diag_smem)) ||
      (rc = allow_smem((const void*)op->ks.rhs, op->ks.rhs_smem)))
    return bail(rc);

  // host tables
  std::vector<long double> nodes = basis::gll_nodes(p), gx, gw;
  basis::gauss_rule(q, gx, gw);
  std::vector<double> Bh, Gh;
  basis::lagrange_tables(nodes, gx, Bh, Gh);
  std::vector<double> ph(q), wh(q);
  for (int i = 0; i < q; ++i) { ph[i] = (double)gx[i]; wh[i] = (double)gw[i]; }

  const int64_t nv = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  const int ncomp = form == FEPA_DIFFUSION ? 6 : 1;
  const int64_t q3 = (int64_t)q * q * q;
  if ((rc = dalloc(&op->verts, 3 * nv)) || (rc = dalloc(&op->gmap, E * n * n * n)) ||
      (rc = dalloc(&op->qd, E * ncomp * q3)) || (rc = dalloc(&op->B, (size_t)q * n)) ||
      (rc = dalloc(&op->G, (size_t)q * n)) || (rc = dalloc(&op->pts, q)) || (rc = dalloc(&op->wts, q)) ||
      (rc = dalloc(&op->flag, 1)))
    return bail(rc);
  cudaStream_t s = op->stream;
#define CREATE_TRY(call)                                                                        \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return bail(fail(FEPA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_))); \
  } while (0)
  CREATE_TRY(cudaMemcpyAsync(op->verts, vertices, 3 * nv * sizeof(double), cudaMemcpyHostToDevice, s));
  CREATE_TRY(cudaMemcpyAsync(op->B, Bh.data(), q * n * sizeof(double), cudaMemcpyHostToDevice, s));
  CREATE_TRY(cudaMemcpyAsync(op->G, Gh.data(), q * n * sizeof(double), cudaMemcpyHostToDevice, s));
  CREATE_TRY(cudaMemcpyAsync(op->pts, ph.data(), q * sizeof(double), cudaMemcpyHostToDevice, s));
  CREATE_TRY(cudaMemcpyAsync(op->wts, wh.data(), q * sizeof(double), cudaMemcpyHostToDevice, s));
  CREATE_TRY(cudaMallocHost((void**)&op->st_host_flag, sizeof(int)));
  CREATE_TRY(cudaMemsetAsync(op->flag, 0, sizeof(int), s));
  build_gmap<<<grid_for(E * n * n * n, 256, 148 * 32), 256, 0, s>>>(nx, ny, nz, p, op->gmap);
  g_launches.fetch_add(1);
  geom_qdata<<<grid_for(E * q3, 256, 148 * 32), 256, 0, s>>>(nx, ny, nz, q, op->verts, op->pts, op->wts,
                                                              form == FEPA_DIFFUSION, op->qd, op->flag);
  g_launches.fetch_add(1);
  CREATE_TRY(cudaGetLastError());
  int bad = 0;
  CREATE_TRY(cudaMemcpyAsync(&bad, op->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CREATE_TRY(cudaStreamSynchronize(s));
  if (bad) return bail(fail(FEPA_ERR_MESH, "non-positive Jacobian determinant at a quadrature point"));
#undef CREATE_TRY
  *out = op;
  return FEPA_OK;
}

void fepa_op_destroy(fepa_op* op) { free_op(op); }

int fepa_op_set_vertices(fepa_op* op, const double* vertices, int32_t on_device) {
  if (!op || !vertices) return fail(FEPA_ERR_ARG, "null argument");
  cudaStream_t s = op->stream;
  const int64_t nv = (int64_t)(op->nx + 1) * (op->ny + 1) * (op->nz + 1);
  const int64_t q3 = (int64_t)op->q * op->q * op->q;
  CUDA_TRY(cudaMemcpyAsync(op->verts, vertices, 3 * nv * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(op->flag, 0, sizeof(int), s));
  geom_qdata<<<grid_for(op->E * q3, 256, 148 * 32), 256, 0, s>>>(op->nx, op->ny, op->nz, op->q, op->verts, op->pts,
                                                                  op->wts, op->form == FEPA_DIFFUSION, op->qd, op->flag);
  LAUNCH_CHECK();
  op->inv_diag_valid = false;
  CUDA_TRY(cudaMemcpyAsync(op->st_host_flag, op->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (*op->st_host_flag) return fail(FEPA_ERR_MESH, "non-positive Jacobian determinant at a quadrature point");
  return FEPA_OK;
}

int64_t fepa_op_ndofs(const fepa_op* op) { return op ? op->N : -1; }
int64_t fepa_op_nelems(const fepa_op* op) { return op ? op->E : -1; }
int32_t fepa_op_q1d(const fepa_op* op) { return op ? op->q : -1; }
int32_t fepa_op_dcomps(const fepa_op* op) { return op ? (op->form == FEPA_DIFFUSION ? 6 : 1) : -1; }

int fepa_op_set_stream(fepa_op* op, void* stream) {
  if (!op) return fail(FEPA_ERR_ARG, "op is null");
  op->stream = (cudaStream_t)stream;
  return FEPA_OK;
}

int fepa_op_boundary_dofs(const fepa_op* op, int32_t* dofs, int64_t capacity, int64_t* count) {
  if (!op || !count) return fail(FEPA_ERR_ARG, "null argument");
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
  if (e == cudaSuccess) {
    const int64_t total = op->E * op->n * op->n * op->n;
    flag_gmap<<<grid_for(total, 256, 148 * 32), 256, 0, s>>>(op->nx, op->ny, op->nz, op->p, dmask, op->gmap);
    g_launches.fetch_add(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dmask);
  if (e != cudaSuccess) return fail(FEPA_ERR_CUDA, "set_essential: %s", cudaGetErrorString(e));
  if (op->ess) { cudaFree(op->ess); op->ess = nullptr; }
  op->ess_count = 0;
  if (count > 0) {
    TRY(dalloc(&op->ess, count));
    CUDA_TRY(cudaMemcpy(op->ess, dofs, count * sizeof(int32_t), cudaMemcpyHostToDevice));
    op->ess_count = count;
  }
  op->inv_diag_valid = false;
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
  qp_coords_kernel<<<grid_for(total, 256, 148 * 32), 256, 0, op->stream>>>(op->nx, op->ny, op->nz, op->q, op->verts,
                                                                         op->pts, out);
  LAUNCH_CHECK();
  return FEPA_OK;
}

int fepa_op_apply(fepa_op* op, const double* x, double* y) {
  if (!op || !x || !y) return fail(FEPA_ERR_ARG, "null argument");
  if (x == y) return fail(FEPA_ERR_ARG, "x and y must not alias");
  CUDA_TRY(cudaMemsetAsync(y, 0, op->N * sizeof(double), op->stream));
  return launch_apply(op, x, y, nullptr, op->stream);
}

int fepa_op_diagonal(fepa_op* op, double* diag) {
  if (!op || !diag) return fail(FEPA_ERR_ARG, "null argument");
  return compute_diagonal(op, diag, op->stream);
}

static int rhs_common(fepa_op* op, const double* f_qp, double scale, double* b) {
  cudaStream_t s = op->stream;
  CUDA_TRY(cudaMemsetAsync(b, 0, op->N * sizeof(double), s));
  op->ks.rhs<<<(int)op->E, op->q * op->q, op->ks.rhs_smem, s>>>(op->nx, op->ny, op->verts, op->gmap, op->pts, op->wts,
                                                                 op->B, f_qp, scale, b);
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
  if (!op || !b_host || !x_host) return fail(FEPA_ERR_ARG, "null argument");
  TRY(ensure_workspace(op));
  if (!op->bw) TRY(dalloc(&op->bw, op->N));
  if (!op->xio) TRY(dalloc(&op->xio, op->N));
  double* xd = op->xio;
  cudaStream_t s = op->stream;
  cudaError_t e = cudaMemcpyAsync(op->bw, b_host, op->N * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xd, x_host, op->N * sizeof(double), cudaMemcpyHostToDevice, s);
  int rc = FEPA_OK;
  if (e != cudaSuccess) rc = fail(FEPA_ERR_CUDA, "host copy: %s", cudaGetErrorString(e));
  if (rc == FEPA_OK) rc = run_cg(op, op->bw, xd, rtol, maxit, precond, stats);
  if (rc == FEPA_OK || rc == FEPA_ERR_NOCONV) {
    std::string keep = g_err;
    e = cudaMemcpyAsync(x_host, xd, op->N * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = fail(FEPA_ERR_CUDA, "host copy back: %s", cudaGetErrorString(e));
    else g_err = keep;
  }
  return rc;
}

int fepa_cg_iterations(fepa_op* op, const double* b, double* x, int32_t iters, int32_t precond, fepa_cg_stats* stats) {
  if (iters < 1) return fail(FEPA_ERR_ARG, "iters must be >= 1");
  int rc = run_cg(op, b, x, 0.0, iters, precond, stats);
  return rc;
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
    TRY(compute_diagonal(op, invd, s));  // zeroes invd, then sums the element diagonals
    reciprocal<<<grid_for(N, 256, 148 * 16), 256, 0, s>>>(N, invd, invd);
    LAUNCH_CHECK();
  }
  const double* pinv = precond ? invd : nullptr;
  CUDA_TRY(cudaMemsetAsync(h, 0, N * sizeof(double), s));
  TRY(launch_apply(op, x, h, nullptr, s));
  cg_init<<<rb, RED_THREADS, 0, s>>>(N, b, r, d, h, pinv, st, rtol * rtol, maxit, partials);
  LAUNCH_CHECK();
  // host-driven loop in chunks; every kernel returns at once after the device sets done
  constexpr int CHUNK = 8;
  CgState hs;
  for (;;) {
    for (int k = 0; k < CHUNK; ++k) {
      TRY(launch_apply(op, d, h, &st->done, s));
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
    stats->status = hs.converged ? FEPA_OK : FEPA_ERR_NOCONV;
    stats->b_norm = sqrt(hs.bb);
    stats->rel_residual = hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0;
    stats->precond_norm = sqrt(fabs(hs.rho));
  }
  if (!hs.converged && rtol > 0.0)
    return fail(FEPA_ERR_NOCONV, "CG did not reach rtol %.3g in %d iterations (rel. residual %.3e)", rtol, hs.iter,
                hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0);
  return FEPA_OK;
}
