/*
 * fepa.h -- matrix-free partial-assembly (PA) finite element operators and their
 * Jacobi-preconditioned CG solve, for H1 mass and diffusion on hexahedral meshes,
 * on one NVIDIA B300 (sm_103a).
 *
 * What the calls compute (arXiv 2402.15940):
 *   The operator is the decomposition A = P^T G^T B^T D B G P of Fig. "fig_feod"
 *   (Sec. 3.5).  On one GPU with a conforming mesh P = I.  G maps the global
 *   (L-vector) DOFs to element DOFs (E-vector) and G^T sums them back; B evaluates
 *   values or reference gradients at the quadrature points (Q-vector) by sum
 *   factorisation of the tensor-product basis (Sec. 2.1); D is the pointwise
 *   quadrature-point factor, the only data partial assembly stores (Sec. 2.2,
 *   "Partial Assembly").  Forms: the CEED bake-off operators BP1 (mass) and BP3
 *   (diffusion) named in Sec. 2.2.  The solver is CG with the matrix-free
 *   diagonal as preconditioner (Sec. 2.1), run as fused device kernels with
 *   warp-level dot products (Sec. 2.3).
 *
 * Discretisation (choices the paper leaves open; the same choices as the CPU
 * oracle's readings):
 *   - reference element [0,1]^3; Lagrange basis of order p on the Gauss-Lobatto-
 *     Legendre nodes; Gauss-Legendre quadrature with q points per direction;
 *   - mesh: a conforming hexahedral mesh given by its vertices and element connectivity
 *     (fepa_op_create_hex), or a structured grid of (nx+1)(ny+1)(nz+1) vertices at
 *     arbitrary positions (x index fastest), element (ex,ey,ez) = ex + nx*(ey + ny*ez)
 *     (fepa_op_create); each element is the trilinear map of its 8 corners;
 *   - global DOFs: on a structured grid the (p*nx+1)(p*ny+1)(p*nz+1) node grid, x
 *     fastest; on a connectivity mesh the numbering of fepa_hex_numbering; element-local
 *     DOF a + (p+1)*(b + (p+1)*c);
 *   - mass: D = w*det(J); diffusion: D = w*adj(J)adj(J)^T/det(J) (symmetric 3x3,
 *     6 stored components xx, xy, xz, yy, yz, zz);
 *   - Dirichlet (essential) DOFs: the constrained operator (I-E) A (I-E) + E.
 *
 * Conventions:
 *   - Every int-returning call returns FEPA_OK (0) or a negative FEPA_ERR_* code and
 *     then fepa_last_error() holds a message (thread-local); fepa_solver_poll may also
 *     return FEPA_BUSY (1).  Nothing aborts or traps.
 *   - "device" pointers are CUDA global-memory pointers of the op's device; "host"
 *     pointers are ordinary CPU memory.  The caller owns every buffer it passes in;
 *     the library owns the fepa_op handle and the device arrays inside it.
 *   - All device work is enqueued on the op's stream (given at creation, may be 0 for
 *     the legacy default stream) and is asynchronous with respect to the host unless
 *     a call says otherwise.
 *   - Values in memory are IEEE binary64 unless a call says otherwise (the FP32 calls take
 *     binary32).  The arithmetic of the "FP64" action (fepa_op_apply and the FP64 solves)
 *     is chosen per op by fepa_op_set_f64_variant: native binary64, or double-float pairs
 *     on the FP32 pipe (about 48 significant bits, relative error far below the 1e-12 of the
 *     action's contract).  That action rescales its input by exact powers of two wherever
 *     the values or their products with D would leave the float exponent range, so it holds
 *     for any finite FP64 input.  The set-up (geometry, D, diagonal, load vector) is also
 *     double-float: an element of extent h must satisfy h >= 2^-20, |coordinates| <= 2^20 and
 *     |coordinates| <= 2^10 h (D then accurate to ~2^-48 |x|/h, 1e-13 on unit-cube meshes up to
 *     256 elements per side); outside that range creation returns FEPA_ERR_UNSUPPORTED.
 */
#ifndef FEPA_H
#define FEPA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FEPA_OK 0
#define FEPA_ERR_ARG (-1)         /* invalid argument (null pointer, size, order ...) */
#define FEPA_ERR_OOM (-2)         /* device allocation failed */
#define FEPA_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define FEPA_ERR_MESH (-4)        /* non-positive Jacobian determinant at a quadrature point */
#define FEPA_ERR_NOCONV (-5)      /* CG reached maxit before the tolerance */
#define FEPA_ERR_TIMEOUT (-6)     /* a kernel's bounded wait for staged data expired (no fault) */
#define FEPA_ERR_UNSUPPORTED (-7) /* order / quadrature outside the compiled range */
#define FEPA_ERR_NONFINITE (-8)   /* a solve's residual norm became NaN or infinite (non-finite b, x or
                                     operator data); the loop stops at once instead of running to maxit */

#define FEPA_BUSY 1               /* fepa_solver_poll: work still in flight */

/* bilinear forms */
#define FEPA_MASS 0       /* BP1: (u, v) */
#define FEPA_DIFFUSION 1  /* BP3: (grad u, grad v) */

/* preconditioners */
#define FEPA_PRECOND_NONE 0
#define FEPA_PRECOND_JACOBI 1

/* how CG iterations are driven (fepa_op_set_cg_mode) */
#define FEPA_CG_GRAPH 0   /* one CUDA graph with a device-side while-condition (default) */
#define FEPA_CG_STREAM 1  /* host-driven chunks of stream launches, state checked per chunk */

/* compiled range: 1 <= p <= FEPA_MAX_ORDER, q = p+1 .. p+2 (q1d > p) */
#define FEPA_MAX_ORDER 8

typedef struct fepa_op fepa_op; /* opaque: mesh + H1 space + form + stored D */

typedef struct fepa_cg_stats {
  int32_t iterations;     /* operator applications inside the loop */
  int32_t status;         /* FEPA_OK, FEPA_ERR_NOCONV or FEPA_ERR_NONFINITE */
  double rel_residual;    /* ||r_k||_2 / ||b||_2 at exit */
  double precond_norm;    /* sqrt(z_k . r_k) at exit (preconditioned residual norm) */
  double b_norm;          /* ||b||_2 */
} fepa_cg_stats;

typedef struct fepa_refine_stats {
  int32_t outer_iterations;  /* FP64 residual corrections applied */
  int32_t inner_iterations;  /* FP32 CG iterations, summed over the corrections */
  int32_t status;            /* FEPA_OK, FEPA_ERR_NOCONV or FEPA_ERR_NONFINITE */
  double rel_residual;       /* ||b - A x||_2 / ||b||_2 with the FP64 operator, at exit */
  double b_norm;             /* ||b||_2 */
} fepa_refine_stats;

/* Version string of the library build. */
const char* fepa_version(void);

/* Thread-local message describing the last error returned on this thread. */
const char* fepa_last_error(void);

/* Number of this library's kernel launches so far in this process (graph-launched
 * kernels included, counted by executed iterations).  Used to attribute GPU work. */
int64_t fepa_launch_count(void);

/*
 * Create an operator on the current CUDA device.
 *   nx, ny, nz    elements per direction (>= 1)
 *   vertices      host, ((nx+1)*(ny+1)*(nz+1)) x 3 doubles, row-major, x index fastest
 *   p             polynomial order, 1..FEPA_MAX_ORDER
 *   q1d           Gauss points per direction; 0 selects p+2; allowed p+1 or p+2
 *   form          FEPA_MASS or FEPA_DIFFUSION
 *   stream        cudaStream_t (as void*) on which all work of this op is enqueued
 * Builds G (element->DOF map), the 1D tables of B, and D (Sec. 2.2, partial
 * assembly: the quadrature-point data is computed once and stored).  Blocks until D
 * is built and returns FEPA_ERR_MESH if any det(J) <= 0, FEPA_ERR_UNSUPPORTED if an element
 * is outside the set-up's range (see the conventions above).  No essential DOFs are set.
 */
int fepa_op_create(int32_t nx, int32_t ny, int32_t nz, const double* vertices, int32_t p, int32_t q1d,
                   int32_t form, void* stream, fepa_op** out);

/*
 * Create an operator on a conforming hexahedral mesh given by its element connectivity, on
 * the current CUDA device: the problem statement of Fig. "fig_feod" (Sec. 3.5), where the mesh
 * defines the global (L-vector) numbering and so G.
 *   nverts, vertices   host, nverts x 3 doubles (row-major)
 *   nelems, conn       host int32 [nelems][8]: the vertex ids of each element in tensor-product
 *                      corner order, corner (i, j, k) of the reference cube at entry i + 2j + 4k
 *                      (i along the first reference direction); any element order, any vertex
 *                      numbering, any orientation of each element (det J > 0 required)
 *   p, q1d, form, stream as fepa_op_create
 * The DOFs are numbered on the host by fepa_hex_numbering's rule; the boundary (for
 * fepa_op_boundary_dofs) is every node on a face that only one element holds.  Returns
 * FEPA_ERR_MESH for a vertex id out of range, an element with a repeated vertex, a face held by
 * more than two elements, two elements whose four common vertices form different
 * quadrilaterals, or det J <= 0 at a quadrature point.  Blocks until D is built.  Every other
 * call takes an op made here as it takes a structured one; fepa_op_set_vertices then takes
 * nverts x 3 doubles.
 */
int fepa_op_create_hex(int64_t nverts, const double* vertices, int64_t nelems, const int32_t* conn, int32_t p,
                       int32_t q1d, int32_t form, void* stream, fepa_op** out);

/*
 * Host only (no device work): the global DOF numbering fepa_op_create_hex uses for order p on
 * the connectivity mesh (nverts, nelems, conn as there), so a caller can map its own data to
 * the op's DOFs.  Each element's local node (a, b, c) is classed as a vertex, edge, face or
 * interior node.  Shared edge and face nodes are placed in a frame every element agrees on:
 * along an edge from its smaller global vertex id; on a face from its smallest-id vertex, the
 * first axis toward the smaller-id of that vertex's two neighbours on the face.  Numbers are
 * handed out vertex by vertex, edge by edge (p-1 each), face by face ((p-1)^2 each) and element
 * interior by element interior ((p-1)^3 each), in the order the elements (in the given order,
 * nodes in local order) first reach them.
 *   elem_dofs   host int32 [nelems][(p+1)^3] receiving G, or null
 *   ndofs       receives the number of global DOFs
 * Errors as fepa_op_create_hex (FEPA_ERR_MESH for an invalid connectivity).
 */
int fepa_hex_numbering(int64_t nverts, int64_t nelems, const int32_t* conn, int32_t p, int32_t* elem_dofs,
                       int64_t* ndofs);

/*
 * Move the mesh: replace the vertex coordinates (same mesh topology) and rebuild D.
 *   vertices     the op's vertex count x 3 doubles (structured: (nx+1)*(ny+1)*(nz+1)),
 *                host or device memory
 *   on_device    0: vertices is a host pointer; 1: a device pointer
 * Blocks until D is rebuilt; returns FEPA_ERR_MESH (D then undefined) if any
 * det(J) <= 0, FEPA_ERR_UNSUPPORTED (D undefined) outside the set-up's range.  Invalidates
 * the cached diagonal.
 */
int fepa_op_set_vertices(fepa_op* op, const double* vertices, int32_t on_device);

/* Release the op and every device array it owns (synchronises its stream). */
void fepa_op_destroy(fepa_op* op);

/* Sizes: global DOFs N, elements E, q1d, number of stored D components per
 * quadrature point (1 mass, 6 diffusion). */
int64_t fepa_op_ndofs(const fepa_op* op);
int64_t fepa_op_nelems(const fepa_op* op);
int32_t fepa_op_q1d(const fepa_op* op);
int32_t fepa_op_dcomps(const fepa_op* op);

/* Change the stream subsequent work of this op is enqueued on. */
int fepa_op_set_stream(fepa_op* op, void* stream);

/* Select how CG iterations are driven: FEPA_CG_GRAPH (default; no host wait per
 * iteration) or FEPA_CG_STREAM (plain stream launches, e.g. for per-kernel profiling).
 * Both run the same kernels and give the same iterates. */
int fepa_op_set_cg_mode(fepa_op* op, int32_t mode);

/* FP32 inner CG of the mixed solves (fepa_solve_refined, fepa_solve_reliable and the
 * refined resumable solve): with enable != 0 (the default) the FP32 action kernel also
 * forms (d, A d) = sum over elements of d_e . (A_e d_e) plus d_g^2 at essential DOFs
 * (Sec. 2.3: the dot product fused into the operator kernel), summed in FP32 per warp and
 * added into 256 doubles, and the separate (d, h) pass over two N-vectors is dropped.  Used where the chosen FP32 variant has that build (p >= 3, variants 0-2);
 * elsewhere, and with enable = 0, (d, h) is a separate reduction.  The two agree to FP32
 * rounding of the element results, not bitwise.  Returns FEPA_ERR_ARG for a null op. */
int fepa_op_set_fused_dot(fepa_op* op, int32_t enable);

/* Boundary DOFs (structured: of the node grid; connectivity mesh: on faces held by one
 * element), ascending, written to dofs (host, capacity entries); *count receives the total
 * (which may exceed capacity: then nothing is written and FEPA_ERR_ARG is returned). dofs
 * may be null to query the count. */
int fepa_op_boundary_dofs(const fepa_op* op, int32_t* dofs, int64_t capacity, int64_t* count);

/* Set the essential (Dirichlet) DOF list (host, count entries, each in [0,N)).
 * Replaces any previous list; count = 0 clears it.  Synchronous. */
int fepa_op_set_essential(fepa_op* op, const int32_t* dofs, int64_t count);

/* Copy of G: element-local to global DOF map, device int32 [E][(p+1)^3]
 * (essential DOFs appear unflagged). */
int fepa_op_elem_dofs(const fepa_op* op, int32_t* out);

/* Copy of D: device double [E][dcomps][q^3], quadrature point i + q*(j + q*k). */
int fepa_op_qdata(const fepa_op* op, double* out);

/* Physical coordinates of the quadrature points: device double [E][q^3][3]. */
int fepa_op_qp_coords(const fepa_op* op, double* out);

/*
 * y = A x (Fig. fig_feod: G^T B^T D B G), with the constrained form
 * y = (I-E) A (I-E) x + E x when essential DOFs are set.
 *   x, y   device, N doubles each; must not overlap.
 */
int fepa_op_apply(fepa_op* op, const double* x, double* y);

/*
 * The same action in FP32: D, the 1D tables, the contractions, x and y are single
 * precision (the operator of the mixed-precision solve).  x, y: device, N floats each.
 * The first call builds an FP32 copy of D (4 bytes per stored value, each component
 * padded to a multiple of 4 values).  The kernel stages each block's D with one TMA
 * bulk copy; if that copy's bounded wait expires the block skips its work and sets an
 * error word that the next blocking call on this op (fepa_solve_refined, fepa_solve_reliable,
 * fepa_solver_poll at the end of a refined solve, fepa_mg_solve with an FP32 V-cycle) reports
 * as FEPA_ERR_TIMEOUT.  The word is cleared when it is reported, so each expiry is reported
 * once.
 */
int fepa_op_apply_f32(fepa_op* op, const float* x, float* y);

/*
 * y = A x in FP32 as fepa_op_apply_f32, and *xax = (x, A x) (xax: one device double),
 * the sum over elements of x_e . (A_e x_e) with x_e zero at essential DOFs, plus x_g^2
 * at each essential DOF: the fused (d, A d) of the FP32 CG (fepa_op_set_fused_dot), the
 * dot product of Sec. 2.3 formed inside the operator kernel.  Where the op's FP32 variant
 * has no such build (p < 3, variant 3) the product is a separate pass over x and y.
 * Enqueued on the op's stream; *xax is valid when that work completes.  Calls on one op
 * share its (x, A x) accumulators: they must not overlap on the GPU (for instance two calls
 * on different streams after fepa_op_set_stream while the first is still running).
 */
int fepa_op_apply_f32_dot(fepa_op* op, const float* x, float* y, double* xax);

/*
 * Launch shape of the FP32 kernel.  Variants: 0 = D staged into shared memory by a TMA
 * bulk copy, 1 = D read directly from HBM (smaller blocks, more warps per SM), 2 = as 1
 * with half as many elements per block, 3 = persistent blocks pipelined over element
 * groups (TMA copy of the next group's D and cp.async gather of its x overlap the
 * current group's arithmetic).  By default (variant -1) the first FP32 use
 * times every variant on this op's mesh, in the form the FP32 CG loop launches it (with
 * (x, A x) fused where the variant has that build and fused products are enabled, else
 * with the separate dot-product pass), in three rounds, each variant's best round
 * counting, and keeps the fastest; the choice is cached per device, (p, q, form) and mesh
 * size class (E < 1e3, 1e4, 1e5, larger) for the process.  All variants compute the same
 * result (up to the order of the atomic additions); their contractions issue two FP32
 * multiply-adds per packed instruction where that measured faster for the (p, q, form).
 */
int fepa_op_set_f32_variant(fepa_op* op, int32_t variant);
int32_t fepa_op_f32_variant(const fepa_op* op);          /* -1 until chosen */
const char* fepa_f32_variant_name(int32_t variant);

/*
 * Arithmetic of the FP64 action (fepa_op_apply and every FP64 solve on this op).
 * Variants: 0 = native FP64 (DFMA), 1 = double-float: x is split into two floats
 * (hi + lo) as it is gathered and D is read as (hi, lo) pairs (a copy of D kept beside
 * the FP64 one, 8 bytes per value), every contraction step is an accurate dot-product
 * step on the FP32 pipe (exact FMA product, TwoSum accumulation, ~2^-48 relative error;
 * the even/odd halves of output pairs in packed two-wide instructions, bit-identical per
 * component), and the element result is recombined in FP64 -- error far inside the FP64
 * action's tolerance.  Each block checks the exponents of its gathered x against D's largest
 * exponent (found by the geometry kernel) and, where the products would leave the
 * float range less the low word's 24 bits, re-gathers x times an exact power of two and
 * scales the results back (a second pass over the block's x, rare).  This library's own
 * design for a GPU whose FP64 rate is a small fraction of its FP32 rate; the paper's
 * FP64 kernels have no counterpart.  2 = the double-float kernel in blocks of half as many
 * elements (the same arithmetic per element; only the order of the atomic additions of the
 * scatter differs; more and smaller blocks, which can fill the GPU better on small meshes).  By default (-1) the first FP64 use times the three
 * on this op's mesh (three rounds, best round each) and keeps the fastest; cached per device,
 * (p, q, form) and mesh size class.  The allocation-free solve never times: it uses the chosen or forced variant
 * (the double-float one only if its copy of D is current), else 0.
 */
int fepa_op_set_f64_variant(fepa_op* op, int32_t variant);
int32_t fepa_op_f64_variant(const fepa_op* op);          /* -1 until chosen */
const char* fepa_f64_variant_name(int32_t variant);

/* diag(A) (of the constrained operator: 1 on essential rows), computed without
 * assembling A by sum factorisation (Sec. 2.1).  diag: device, N doubles. */
int fepa_op_diagonal(fepa_op* op, double* diag);

/* b = G^T B^T (w det(J) f): load vector of f given at the quadrature points.
 *   f_qp  device double [E][q^3]; b device, N doubles (overwritten).
 * Computed in double-float: |f| w det J should stay within 2^-70 .. 2^100 where it matters.
 * Essential rows are left as computed (the caller sets boundary values). */
int fepa_op_rhs(fepa_op* op, const double* f_qp, double* b);

/* As fepa_op_rhs with f = scale * sin(pi x) sin(pi y) sin(pi z) evaluated in-kernel
 * at the physical quadrature points, and essential rows of b set to 0
 * (homogeneous Dirichlet data, the manufactured problem). */
int fepa_op_rhs_sine(fepa_op* op, double scale, double* b);

/*
 * Solve A x = b by CG, preconditioned with diag(A) (FEPA_PRECOND_JACOBI) or not.
 *   b      device, N doubles
 *   x      device, N doubles: initial guess on entry, solution on exit
 *   rtol   stop when ||r_k||_2 <= rtol * ||b||_2
 *   maxit  iteration limit (>= 1)
 *   stats  host, may be null
 * Iterations run on the device inside one CUDA graph with a device-side loop
 * condition; the call blocks until the solve ends.  Returns FEPA_ERR_NOCONV (with
 * stats filled and x holding the last iterate) if maxit is reached first.
 */
int fepa_cg_solve(fepa_op* op, const double* b, double* x, double rtol, int32_t maxit, int32_t precond,
                  fepa_cg_stats* stats);

/* As fepa_cg_solve with HOST b and x (N doubles each): copies b and x to the device,
 * solves, copies x back; blocks until done. */
int fepa_cg_solve_host(fepa_op* op, const double* b_host, double* x_host, double rtol, int32_t maxit,
                       int32_t precond, fepa_cg_stats* stats);

/*
 * Fixed-count CG iterations (no stopping test) for timing the per-iteration cost:
 * runs exactly `iters` iterations from x (device), preconditioned like fepa_cg_solve.
 * stats->rel_residual holds the residual after them.  Blocks until done.
 */
int fepa_cg_iterations(fepa_op* op, const double* b, double* x, int32_t iters, int32_t precond,
                       fepa_cg_stats* stats);

/*
 * Mixed-precision solve: FP64 iterative refinement around an FP32 Jacobi-PCG.
 * Each outer step forms r = b - A x with the FP64 operator and FP64 reductions; when
 * ||r||_2 > rtol ||b||_2 it solves A e = r with the FP32 operator (fepa_op_apply_f32)
 * to relative residual inner_rtol (at most inner_maxit iterations; FP32 vectors, dot
 * products accumulated to FP64 accuracy, except (d, A d), which by default comes out of the
 * FP32 action kernel (fepa_op_set_fused_dot); FP64 scalars) and updates x += e in FP64.
 * When less than inner_rtol is enough to reach rtol (the last correction) the inner
 * tolerance is relaxed to 0.25 rtol ||b|| / ||r||, at most 0.5.  A residual whose norm has a
 * binary exponent beyond +-20 enters the FP32 solve scaled by an exact power of two (and the
 * correction is scaled back), so problems of any FP64 magnitude keep the FP32 loop in range.
 *   b, x        device, N doubles (x: initial guess in, solution out)
 *   rtol        outer stopping rule on the FP64 residual
 *   max_outer   limit on corrections; FEPA_ERR_NOCONV (stats filled) if reached
 * Blocks until done.  The essential set and preconditioner are those of fepa_cg_solve.
 */
int fepa_solve_refined(fepa_op* op, const double* b, double* x, double rtol, int32_t max_outer, double inner_rtol,
                       int32_t inner_maxit, int32_t precond, fepa_refine_stats* stats);

/*
 * Mixed-precision CG with reliable updates (residual replacement): a single FP32
 * Jacobi-PCG recurrence (FP32 operator and vectors, dot products to FP64 accuracy or, for
 * (d, A d), fused into the FP32 action (fepa_op_set_fused_dot); FP64 scalars) whose residual is replaced by the FP64 residual b - A x (FP64 operator and
 * reductions) each time it has fallen by the factor delta since the last replacement;
 * the FP32 iterate is added to the FP64 x first.  The search direction and scalars
 * carry over each replacement, so unlike fepa_solve_refined the Krylov space is kept and
 * the iteration count stays close to the FP64 solve's.  This library's own addition
 * (a standard mixed-precision CG technique); the paper describes no mixed-precision
 * solver.
 *   delta   replacement factor in (0, 1); 0.01-0.3 measured within 5 % of each other on
 *           BP3 (0.03 best); below 1e-3 the FP32 recurrence drifts and convergence stalls
 *   maxit   limit on FP32 iterations in total; FEPA_ERR_NOCONV (stats filled) if reached
 * Stops when ||b - A x||_2 <= rtol ||b||_2 with the FP64 operator.  stats: outer_iterations
 * = replacements, inner_iterations = FP32 iterations.  The FP32 recurrence works in units of
 * a power of two fixed at the first residual (as fepa_solve_refined scales its residuals).
 * Blocks until done.
 */
int fepa_solve_reliable(fepa_op* op, const double* b, double* x, double rtol, double delta, int32_t maxit,
                        int32_t precond, fepa_refine_stats* stats);
int fepa_solve_reliable_host(fepa_op* op, const double* b_host, double* x_host, double rtol, double delta,
                             int32_t maxit, int32_t precond, fepa_refine_stats* stats);

/* As fepa_solve_refined with HOST b and x (copies inside the call). */
int fepa_solve_refined_host(fepa_op* op, const double* b_host, double* x_host, double rtol, int32_t max_outer,
                            double inner_rtol, int32_t inner_maxit, int32_t precond, fepa_refine_stats* stats);

/* ---------------------------------------------------------------------------
 * Resumable solves, for schedulers that keep many problems resident and interleave
 * their iterations (continuous batching): start a solve, enqueue bounded numbers of
 * iterations on the op's stream, and poll for completion without blocking.  Each op
 * runs at most one resumable solve at a time; b and x must stay valid until it ends.
 * Results equal those of fepa_cg_solve / fepa_solve_refined on the same op.
 * ------------------------------------------------------------------------- */
#define FEPA_SOLVER_CG 0       /* FP64 (Jacobi-)PCG */
#define FEPA_SOLVER_REFINED 1  /* FP64 iterative refinement around FP32 PCG */

typedef struct fepa_solver_state {
  int32_t done;              /* 1 once the solve has ended (x holds the result) */
  int32_t status;            /* FEPA_OK or FEPA_ERR_NOCONV when done */
  int32_t iterations;        /* CG iterations so far (inner FP32 ones for REFINED) */
  int32_t outer_iterations;  /* corrections applied (REFINED) */
  double rel_residual;       /* latest ||r|| / ||b|| (FP64 residual for REFINED) */
} fepa_solver_state;

/*
 * Start a resumable solve on the op's stream (asynchronous).
 *   kind        FEPA_SOLVER_CG or FEPA_SOLVER_REFINED
 *   b, x        device, N doubles; x holds the initial guess and, once done, the solution
 *   rtol        stopping rule (FP64 residual)
 *   maxit       CG iteration limit (REFINED: per inner solve)
 *   max_outer   REFINED: limit on corrections (ignored for CG)
 *   inner_rtol  REFINED: inner relative tolerance in (0,1) (ignored for CG)
 */
int fepa_solver_start(fepa_op* op, int32_t kind, const double* b, double* x, double rtol, int32_t maxit,
                      int32_t max_outer, double inner_rtol, int32_t precond);

/* Enqueue up to `iterations` more CG iterations (asynchronous; no-op between phases). */
int fepa_solver_advance(fepa_op* op, int32_t iterations);

/*
 * Check progress.  blocking = 0: returns FEPA_BUSY while the enqueued work is still in
 * flight; otherwise fills *state, and for REFINED enqueues the next phase (correction
 * and FP64 residual, or the next inner solve) when one has finished.
 */
int fepa_solver_poll(fepa_op* op, int32_t blocking, fepa_solver_state* state);

/* ---------------------------------------------------------------------------
 * Batches of independent problems.  Each problem i is its own structured hex mesh,
 * order and form; the batch owns one concatenated DOF vector (problem i occupies
 * [off_i, off_{i+1})), so its operator is block diagonal.  Problems with equal
 * (p, q = p+2, form) share one fused-kernel launch per action; the CG solve advances
 * every problem at once with per-problem scalars, stopping rule and iteration count,
 * skips problems that have converged, and runs as one CUDA graph (while-node) until the
 * last problem stops.  The paper's operator and solver (Fig. fig_feod, Sec. 2.1, 2.3)
 * applied to many small problems, where launch count and tail effects decide the
 * throughput (the strong-scaling concern of Sec. 2.3).
 * ------------------------------------------------------------------------- */
typedef struct fepa_batch fepa_batch;

typedef struct fepa_batch_stats {
  int32_t max_iterations;   /* iterations of the slowest problem */
  int32_t converged;        /* problems that reached rtol */
  int32_t status;           /* FEPA_OK when all did, else FEPA_ERR_NOCONV */
  int32_t reserved;
  double dof_iterations;    /* sum over problems of N_i * iterations_i */
  double max_rel_residual;  /* largest ||r_i|| / ||b_i|| at exit */
} fepa_batch_stats;

/*
 * Create a batch on the current device.
 *   count               number of problems (>= 1)
 *   dims                host int32 [count][3]: nx, ny, nz of each problem
 *   vertices            host array of count host pointers; problem i's vertex grid as in
 *                       fepa_op_create ((nx+1)(ny+1)(nz+1) x 3 doubles)
 *   orders, forms       host int32 [count]: p (1..FEPA_MAX_ORDER) and FEPA_MASS/DIFFUSION
 *   essential_boundary  1: every diffusion problem fixes all its boundary DOFs
 *   stream              cudaStream_t (as void*)
 * q = p+2 for every problem.  Blocks until the data is built.
 */
int fepa_batch_create(int32_t count, const int32_t* dims, const double* const* vertices, const int32_t* orders,
                      const int32_t* forms, int32_t essential_boundary, void* stream, fepa_batch** out);
void fepa_batch_destroy(fepa_batch* batch);
int64_t fepa_batch_ndofs(const fepa_batch* batch);                   /* total DOFs */
int fepa_batch_offsets(const fepa_batch* batch, int64_t* offsets);   /* host, count + 1 entries */
int32_t fepa_batch_groups(const fepa_batch* batch);                  /* distinct (p, form) */
/* The autotuner's picks for group `group` (0 .. groups-1; groups in order of first appearance
 * of their (p, form)): order, form, elements, FP64 action variant (as fepa_batch_set_f64_variant;
 * -1 until the first FP64 apply or solve chose it) and the FP32 tile's elements per block (0 until
 * the first refined or reliable solve chose it).  Outputs may be null. */
int fepa_batch_group_info(const fepa_batch* batch, int32_t group, int32_t* order, int32_t* form, int64_t* elements,
                          int32_t* f64_variant, int32_t* f32_elems_per_block);
int fepa_batch_set_stream(fepa_batch* batch, void* stream);

/* FP64 action variant of every group (as fepa_op_set_f64_variant: 0 DFMA, 1 double-float,
 * 2 double-float in half-size tiles -- the elements per block of the group's persistent
 * kernel; -1 = the process-wide choice for the group's (p, q, form, size class) if one was
 * measured, else the fastest of the three timed on the group at the next apply or solve). */
int fepa_batch_set_f64_variant(fepa_batch* batch, int32_t variant);

/* y = A x for every problem at once (x, y: device, total DOFs). */
int fepa_batch_apply(fepa_batch* batch, const double* x, double* y);

/*
 * Solve every problem by (Jacobi-)PCG as fepa_cg_solve does, all at once.
 *   b, x        device, total DOFs (x: initial guesses in, solutions out)
 *   iterations  host int32 [count] receiving each problem's iteration count (may be null)
 * Blocks until the last problem stops; FEPA_ERR_NOCONV if any problem hit maxit.
 */
int fepa_batch_solve(fepa_batch* batch, const double* b, double* x, double rtol, int32_t maxit, int32_t precond,
                     fepa_batch_stats* stats, int32_t* iterations);

typedef struct fepa_batch_refine_stats {
  int32_t max_inner_iterations;  /* FP32 iterations of the problem that needed the most (all steps) */
  int32_t converged;             /* problems whose FP64 residual reached rtol */
  int32_t status;                /* FEPA_OK when all did, else FEPA_ERR_NOCONV */
  int32_t outer_iterations;      /* refinement steps taken (FP32 correction solves) */
  double dof_iterations;         /* sum over problems of N_i * FP32 iterations_i */
  double max_rel_residual;       /* largest FP64 ||b_i - A x_i|| / ||b_i|| at exit */
} fepa_batch_refine_stats;

/*
 * Mixed-precision solve of every problem, all at once: FP64 iterative refinement around
 * FP32 Jacobi-PCG corrections, as fepa_solve_refined does for one operator, over the
 * batch of fepa_batch_solve (the operator and solver of Fig. fig_feod, Sec. 2.1, 2.3;
 * the mixed precision is this library's addition).
 * Each step computes every problem's FP64 residual b_i - A x_i with the FP64 action;
 * problems at ||r_i|| <= rtol ||b_i|| are finished and do no further work (their elements
 * are skipped by the FP32 action); the others solve A e_i = r_i in FP32 to relative
 * tolerance inner_rtol (relaxed on a problem's last step to what reaching rtol needs) or
 * inner_maxit iterations, in one CUDA-graph loop over the batch, and x_i += e_i.
 *   b, x        device, total DOFs (x: initial guesses in, solutions out, updated in place)
 *   iterations  host int32 [count]: FP32 iterations of each problem over all steps (may be null)
 * The first call builds an FP32 copy of every group's D (half the FP64 D's size).  Unlike
 * fepa_solve_refined the residuals enter the FP32 loop unscaled: each problem's residual
 * entries and their products should stay within the float range (about 1e-18 .. 1e18).
 * FEPA_ERR_NOCONV if a problem has not reached rtol after max_outer steps;
 * FEPA_ERR_TIMEOUT if an FP32 action kernel gave up its bounded wait.
 */
int fepa_batch_solve_refined(fepa_batch* batch, const double* b, double* x, double rtol, int32_t max_outer,
                             double inner_rtol, int32_t inner_maxit, int32_t precond,
                             fepa_batch_refine_stats* stats, int32_t* iterations);

/*
 * Mixed-precision CG with reliable updates for every problem at once, as fepa_solve_reliable
 * does for one operator: one FP32 Jacobi-PCG recurrence per problem (per-problem scalars and
 * stops, one CUDA-graph loop over the batch) whose residual is replaced by the FP64 residual
 * b_i - A x_i each time it has fallen by delta since the last replacement, the FP32 iterate
 * being added to the FP64 x first; directions and scalars carry over each replacement.  The
 * batch steps together: a replacement happens when every problem still running has reached
 * its segment end.  Problems at ||r_i|| <= rtol ||b_i|| drop out (their elements are skipped).
 *   delta       replacement factor in (0, 1)
 *   maxit       limit on each problem's FP32 iterations in total
 *   stats       outer_iterations = replacements, max_inner_iterations = the largest FP32 count
 *   iterations  host int32 [count]: each problem's FP32 iterations (may be null)
 * FEPA_ERR_NOCONV if a problem has not reached rtol within maxit FP32 iterations.
 */
int fepa_batch_solve_reliable(fepa_batch* batch, const double* b, double* x, double rtol, double delta,
                              int32_t maxit, int32_t precond, fepa_batch_refine_stats* stats,
                              int32_t* iterations);

/* ---------------------------------------------------------------------------
 * p-multigrid preconditioner (Sec. 2.1: a hierarchy of orders on one mesh, transfers
 * between them by sum factorisation, diagonal-based smoothers with Chebyshev
 * acceleration).  Levels p, max(1, p/2), ..., 1 built from the fine op's mesh and form;
 * essential DOFs must be none or exactly the boundary (each level then fixes its own
 * boundary).  Smoother: `smooth_degree` Chebyshev-Jacobi steps on
 * [0.245, 1.08] * lambda_max(D^{-1}A) (10 Lanczos steps at set-up); coarsest level:
 * `coarse_degree` steps on [0.003, 1.18] * lambda_max.  The V-cycle is symmetric and
 * linear, so it preconditions plain CG.  precision: FEPA_MG_FP64, or FEPA_MG_FP32 for an
 * FP32 V-cycle (FP32 operators, smoothers and transfers on every level) inside the FP64
 * CG (whose operator action, dot products and scalars stay FP64).  The fine op must
 * outlive the object.
 * ------------------------------------------------------------------------- */
typedef struct fepa_mg fepa_mg;
#define FEPA_MG_FP64 0
#define FEPA_MG_FP32 1

int fepa_mg_create(fepa_op* fine, int32_t smooth_degree, int32_t coarse_degree, int32_t precision, fepa_mg** out);
/* After fepa_op_set_vertices on the fine op: move every level's mesh and rebuild its
 * diagonal and lambda_max (no allocation).  FEPA_ERR_ARG while a resumable solve
 * (fepa_mg_solver_start) has not finished. */
int fepa_mg_update(fepa_mg* mg);
void fepa_mg_destroy(fepa_mg* mg);
int32_t fepa_mg_levels(const fepa_mg* mg);
/* order, DOFs and lambda_max(D^{-1}A) estimate of a level (0 = finest); outputs may be null */
int fepa_mg_level_info(const fepa_mg* mg, int32_t level, int32_t* order, int64_t* ndofs, double* lambda_max);
/* x_level = P x_{level+1} (device vectors of the two levels' sizes); FP64 V-cycle only */
int fepa_mg_prolong(fepa_mg* mg, int32_t level, const double* x_coarse, double* x_fine);
/* r_{level+1} = P^T r_level, coarse essential rows set to 0; FP64 V-cycle only */
int fepa_mg_restrict(fepa_mg* mg, int32_t level, const double* r_fine, double* r_coarse);
/* x = S b with the level's Chebyshev smoother (coarse solver on the last level), from 0;
 * FP64 V-cycle only */
int fepa_mg_smooth(fepa_mg* mg, int32_t level, const double* b, double* x);
/* x = M^{-1} b, one V-cycle on the finest level (FP64 b, x in either precision mode) */
int fepa_mg_vcycle(fepa_mg* mg, const double* b, double* x);
/* CG on the fine op preconditioned by the V-cycle (flexible Polak-Ribiere beta, equal to
 * the standard one for an exact fixed preconditioner); blocks until done */
int fepa_mg_solve(fepa_mg* mg, const double* b, double* x, double rtol, int32_t maxit, fepa_cg_stats* stats);
/* The same solve in resumable form (Sec. 2.1's preconditioned CG, driven by a serving loop as
 * fepa_solver_start/advance/poll drive the Jacobi forms): start enqueues r = b - A x and the
 * stopping threshold on the fine op's stream; advance enqueues up to `iterations` iterations
 * (V-cycle and CG steps; an iteration enqueued after the stopping test has fired changes
 * nothing but runs its V-cycle on the hierarchy's own vectors); poll returns FEPA_BUSY while
 * the last enqueued work runs (blocking = 0) or waits for it, then reads the state, and once
 * done copies the solution into x (device, N doubles, which must stay valid until then).
 * The iterates equal fepa_mg_solve's.  One solve at a time per hierarchy; state.iterations
 * counts CG iterations, outer_iterations is 0. */
int fepa_mg_solver_start(fepa_mg* mg, const double* b, double* x, double rtol, int32_t maxit);
int fepa_mg_solver_advance(fepa_mg* mg, int32_t iterations);
int fepa_mg_solver_poll(fepa_mg* mg, int32_t blocking, fepa_solver_state* state);

/*
 * CG solve that allocates nothing.  The paper has no counterpart: this call exists
 * for callers that cannot allocate device memory once they are running -- for
 * instance a host program whose framework has already reserved the whole GPU for its
 * own caching pool (a cudaMalloc would fail), or a latency-bound loop that must not
 * call cudaMalloc/cudaFree because they can synchronise the device and stall other
 * streams.  fepa_cg_solve, by contrast, allocates its work vectors on first use.
 *
 * Same arguments, result and status codes as fepa_cg_solve; x is iterated in place.
 * The work vectors live in one static device array of this library, sized for at
 * most FEPA_NOALLOC_MAX_DOFS global DOFs (about 4.2 MB, held on every GPU that loads
 * the library until the process exits).  Larger operators are rejected with
 * FEPA_ERR_ARG before any device work.  The iteration loop is driven from the host
 * in short chunks of stream launches (no CUDA graph is built).
 *   - The first call on a device looks up the array's device address (with that
 *     device current); make that first call before any stream capture.
 *   - Every call shares the array and finds it holding the previous call's
 *     contents; the call clears what must start at zero itself.  Calls that overlap
 *     on the GPU (other streams, other threads, other ops) race on the array: run
 *     them one after another.
 */
#define FEPA_NOALLOC_MAX_DOFS 131072
int fepa_cg_solve_noalloc(fepa_op* op, const double* b, double* x, double rtol, int32_t maxit, int32_t precond,
                          fepa_cg_stats* stats);

/*
 * Testing only.  Poll limit of the FIRST bounded wait in the FP32 action kernels that stage
 * D by TMA (variants 0 and 3): the wait of each block for its D copy.  iterations < 0 restores
 * the default (2^22 polls).  With 0 the wait gives up at once: the block skips its work, sets
 * the op's error word and still waits, with the full limit, for its copy in flight before it
 * exits, so the timeout path (FEPA_ERR_TIMEOUT) runs without a fault or a hang.  Applies
 * process-wide to kernels launched on the current device after the call; synchronous.
 */
int fepa_test_set_first_wait_limit(int32_t iterations);

#ifdef __cplusplus
}
#endif

#endif /* FEPA_H */
