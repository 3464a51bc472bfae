/*
 * bem.h -- C ABI of the GB300 panel-interaction library (libbem.so).
 *
 * The library evaluates the indirect single-layer boundary element method of
 * "Dielectric Breakdown Prediction with GPU-Accelerated BEM" (arXiv:2003.12663):
 * a virtual surface charge sigma, piecewise constant on flat triangles
 * (Sec. 3), generates the potential
 *
 *     phi(x) = sum_j u_j S_j(x),   S_j(x) = 1/(4 pi) int_{tau_j} 1/|x-y| dS_y        (Eq. SL)
 *
 * and the field
 *
 *     E(x)   = sum_j u_j G_j(x),   G_j(x) = 1/(4 pi) int_{tau_j} (x-y)/|x-y|^3 dS_y
 *
 * (field formula at the end of Sec. 2).  A pair (x, tau_j) is regular when the
 * distance D from x to the circumcentre of tau_j exceeds eta * R_j, R_j the
 * circumradius (Sec. 4); regular pairs are integrated by a Duffy-transformed
 * Gauss rule with g x g nodes, all other pairs by the closed-form integral of a
 * uniform density over a flat triangle, in FP64.
 *
 * Units: potentials and fields are those of phi = int sigma/(4 pi r); the
 * permittivities are relative values.  Unit normals point out of every body,
 * toward eps_plus; a triangle's vertices are counter-clockwise about its normal.
 *
 * Conventions for every call:
 *  - the return value is a status (BEM_OK or a negative BEM_ERR_*); no call
 *    throws, aborts or exits; bem_last_error() gives a message for the last error;
 *  - "dev" pointers are CUDA device pointers, "host" pointers host memory; all of
 *    them are owned by the caller and are only read or written during the call
 *    (device work is queued on the context's stream and may still be running when
 *    the call returns, except where a call says it synchronises);
 *  - arrays are dense, row-major, in the element type stated;
 *  - a context owns only the precomputed panel data and a fixed workspace sized
 *    at bem_create; the evaluation calls allocate no device memory;
 *  - one context is used by one host thread at a time.
 */
#ifndef BEM_H
#define BEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BEM_OK = 0,
    BEM_ERR_ARG = -1,           /* an argument is out of range or a pointer is NULL */
    BEM_ERR_CUDA = -2,          /* a CUDA runtime call failed */
    BEM_ERR_DEGENERATE = -3,    /* a triangle has zero area */
    BEM_ERR_NOT_CONVERGED = -4, /* the solver stopped at its iteration limit */
    BEM_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up */
    BEM_ERR_NOMEM = -6,         /* a device allocation in bem_create failed */
    BEM_ERR_CAPACITY = -7       /* a size exceeds the workspace fixed at bem_create */
};

/* Boundary condition of a group of triangles (Sec. 2, Eqs. Final1-Final4).
 * BEM_SHEET: a thin floating conductive sheet modelled by a single, possibly open
 * surface (Eq. sheets): potential rows as BEM_FLOATING, neutrality row with the
 * fields of both sides.  Floating conductors and sheets share the floating ids.
 * Field lines end on conductor and floating bodies, which must be closed
 * surfaces; they do not end on sheets. */
enum { BEM_CONDUCTOR = 0, BEM_FLOATING = 1, BEM_DIELECTRIC = 2, BEM_SHEET = 3 };

/* Arithmetic of the regular (far-field) pairs.  BEM_FP64: every step in FP64.
 * BEM_MIXED: regular pairs in FP32 with compensated FP32 accumulation; the
 * closed-form near pairs, reductions and everything else in FP64.
 * BEM_DF (bem_matvec only): the FP64 form's operator with its regular pairs in
 * double-FP32 arithmetic (see BEM_RESIDUAL_DF), agreeing with BEM_FP64 to ~1e-13. */
enum { BEM_FP64 = 0, BEM_MIXED = 1, BEM_DF = 2 };

typedef struct {
    int32_t kind;        /* BEM_CONDUCTOR, BEM_FLOATING, BEM_DIELECTRIC or BEM_SHEET */
    int32_t floating_id; /* BEM_FLOATING, BEM_SHEET: 0 .. n_floating-1, one id per floating body */
    double V0;           /* BEM_CONDUCTOR: prescribed potential (Eq. conductor) */
    double eps_plus;     /* permittivity on the normal's side (Eqs. Jump, Final4, Final3) */
    double eps_minus;    /* BEM_DIELECTRIC, BEM_SHEET: permittivity on the other side
                            (a sheet may take 0, which gives the closed floating body's row) */
} bem_region;

typedef struct {
    int64_t nv;                 /* number of vertices */
    int64_t np;                 /* number of triangles N */
    const double* X;            /* host [nv][3] vertex coordinates */
    const int32_t* tri;         /* host [np][3] vertex indices, CCW about the outward normal */
    const int32_t* region;      /* host [np] index into regions */
    int32_t nregions;
    const bem_region* regions;  /* host [nregions] */
} bem_mesh;

typedef struct {
    double eta;              /* pair is regular iff D > eta R (Sec. 4); default 4 */
    int32_t far_order;       /* g: Duffy/Gauss rule with g x g nodes; 1..6, default 3 */
    int32_t gmres_restart;   /* restart length m of GMRES(m); default 100 */
    int32_t max_iters;       /* total GMRES iteration limit per solve; default 2000 */
    int32_t max_refine;      /* BEM_MIXED: iterative-refinement steps; default 6 */
    int64_t max_points;      /* largest M of one bem_eval_field chunk; default 131072 */
    int32_t timing;          /* != 0: time every regular-pair kernel with CUDA events (bem_counters) */
    int32_t residual;        /* BEM_MIXED refinement residual b - A u: BEM_RESIDUAL_DF_UPDATE
                                (default), BEM_RESIDUAL_DF or BEM_RESIDUAL_FP64 */
    int32_t far32_variant;   /* FP32 regular-pair kernel: 1 scalar, 2, 3 or 4 packed target
                                pairs per thread (3: registers capped for three CTAs per SM);
                                0 (default): bem_create times the candidates on the mesh's own
                                matvec and keeps the fastest (N >= 4096; else 2) */
    int32_t adjoint_checkpoint; /* bem_adjoint keeps the state of every line every this many
                                   RK4 steps and recomputes the steps in between; default 128 */
    int64_t adjoint_lines;   /* lines bem_adjoint holds at once (more are taken in turns); the
                                adjoint workspace (checkpoints for this many lines at the default
                                step limit, one segment of step records, per-line gradient
                                buffers of at most 64 MiB, the transposed operator's near pairs
                                by column) is allocated by bem_create; 0: none (bem_adjoint and
                                bem_matvec_transpose then return BEM_ERR_CAPACITY); default 256 */
    int32_t trace_cluster;   /* CTAs per tracer cluster, 1..8: on meshes of 8192 triangles or
                                more every round's triangles are split over them; 0 (default):
                                chosen per launch from the mesh size and the number of lines
                                (wide clusters for few lines, plain CTAs for many) */
} bem_params;

/* How the iterative refinement of BEM_MIXED forms its residual b - A u.
 * BEM_RESIDUAL_FP64: the FP64 regular-pair kernel.  BEM_RESIDUAL_DF: the same pairs
 * in double-FP32 arithmetic (an unevaluated sum of two floats, error-free
 * transformations of Dekker and Knuth) on the FP32 units, about 1e-13 relative per
 * pair, with the pair classification of the FP64 form reproduced exactly.
 * BEM_RESIDUAL_DF_UPDATE (default): the first residual of a solve in double-FP32; each
 * later one as r - A d, the previous residual less the mixed product of the step's
 * correction d, while |d| <= 1e-3 |u| (else in double-FP32 again).  The product's FP32
 * rounding, about 1e-7 |A| |d|, is then below 1e-10 |A| |u|: the true residual of the
 * result differs from the one the refinement stops on by that much, and the solve
 * needs one double-FP32 pass instead of one per refinement step. */
enum { BEM_RESIDUAL_DF = 0, BEM_RESIDUAL_FP64 = 1, BEM_RESIDUAL_DF_UPDATE = 2 };

/* Work done by a context since creation or the last bem_reset_counters.
 * Index [BEM_FP64] / [BEM_MIXED] / [2] = double-FP32 residual pass. */
typedef struct {
    int64_t kernel_launches;    /* CUDA kernels this library launched */
    int64_t far_launches[3];    /* regular-pair kernel launches */
    int64_t pairs[3];           /* (target, triangle) pairs those launches covered, M x N each */
    int64_t near_pairs[3];      /* of those, pairs classified near and taken by the closed form */
    double far_ms[3];           /* summed regular-pair kernel time in ms (params.timing != 0) */
    int64_t matvecs[3];         /* matrix-free products, solver-internal ones included */
    int64_t gmres_iters;        /* Arnoldi steps */
    int64_t far32_variant;      /* FP32 kernel variant in use (1, 2, 3 or 4; not reset) */
    int64_t phi_pairs[3];       /* of pairs, those of product tiles holding only conductor rows,
                                   summed for phi alone (their row equation needs no E) */
    int64_t chunks32p;          /* 32-triangle chunks the packed FP32 kernel (variants 2-4) staged,
                                   summed over its CTAs */
    int64_t fast_chunks32p;     /* of those, chunks whose every pair with the CTA's targets was
                                   certainly regular (bounding spheres), summed without classification */
} bem_counters;

/* The shape the context's FP32 regular-pair kernel runs with, and how it was chosen
 * (bem_create's tuner: every candidate timed on the mesh's own mixed matvec). */
typedef struct {
    int32_t far32_variant;   /* 1 scalar, 2, 3 or 4 packed target pairs per thread */
    int32_t far32_slots;     /* CTA slots per SM the number of triangle slices aims at */
    int32_t source;          /* 0 fixed (params.far32_variant, or N < 4096), 1 timed by this
                                bem_create, 2 taken from the process-wide table (same device, size
                                bucket and far_order, timed by an earlier context) */
    int32_t bucket;          /* size bucket floor(2 log2 N) */
    int32_t n_candidates;    /* candidates timed (source 1) */
    int32_t cand_variant[12];
    int32_t cand_slots[12];
    float cand_ms[12];       /* one mixed matvec of this mesh per candidate */
} bem_tuning;

typedef struct bem_ctx bem_ctx;

/* Fill p with the defaults above.  Never fails. */
void bem_default_params(bem_params* p);

/*
 * Create a context for one mesh: copies the mesh to the device of the current
 * CUDA device, computes per-triangle geometry and quadrature nodes, the near
 * pairs of every collocation point (centroid) with their closed-form values, and
 * allocates the workspace.  stream: cudaStream_t (NULL = legacy default stream)
 * on which every later call of this context queues its work.  params may be NULL
 * (defaults).  Synchronises the stream before returning.
 * Errors: BEM_ERR_ARG (bad sizes, indices, region data), BEM_ERR_DEGENERATE,
 * BEM_ERR_NOMEM, BEM_ERR_CUDA.  On error *out is NULL.
 */
int bem_create(bem_ctx** out, const bem_mesh* mesh, const bem_params* params, void* stream);

/* Free a context (NULL is allowed).  Synchronises its stream first. */
int bem_destroy(bem_ctx* ctx);

/* Message of the last error on ctx, or of the last failed bem_create if ctx is NULL. */
const char* bem_last_error(const bem_ctx* ctx);

/* Sizes: N triangles, N + n_floating unknowns, n_floating, near pairs of the
 * collocation points (any output pointer may be NULL). */
int bem_sizes(const bem_ctx* ctx, int64_t* n_panels, int64_t* n_unknowns, int64_t* n_floating,
              int64_t* near_pairs);

/* Wait for the context's stream; returns BEM_ERR_TIMEOUT if a device-side wait
 * gave up since the last call, else BEM_OK or BEM_ERR_CUDA. */
int bem_sync(bem_ctx* ctx);

/* Copy the work counters into *out (host).  Synchronises the stream. */
int bem_get_counters(bem_ctx* ctx, bem_counters* out);

/* The tuner's choice for this context (host struct).  Never synchronises. */
int bem_get_tuning(const bem_ctx* ctx, bem_tuning* out);

/* Forget the tuner's process-wide table (the next context of every size bucket times
 * its candidates again). */
void bem_clear_tuning_table(void);

/* Zero the work counters. */
int bem_reset_counters(bem_ctx* ctx);

/*
 * Rows [row0, row1) of the dense collocation matrix A of Eqs. Final1-Final4
 * (Sec. 3: sigma_h = sum_j u_j psi_j, psi_j = 1 on tau_j; equations imposed at
 * the centroids c_i).  The unknowns are u_0..u_{N-1} followed by the potentials
 * V_f of the floating bodies; A is (N+F) x (N+F).  Row i < N with normal n_i:
 *   conductor : A_ij = S_j(c_i)
 *   floating f: A_ij = S_j(c_i),                      A_{i,N+f} = -1
 *   dielectric: A_ij = (eps+ - eps-) n_i.G_j(c_i) + delta_ij (eps+ + eps-)/2
 * Row N+f (charge neutrality of floating body f, Eq. Final4 by the centroid rule,
 * divided by the body's area):  A_{N+f,j} = sum_{i in f} A_i eps+ (delta_ij/2 + n_i.G_j(c_i)) / area_f;
 * rows i of a sheet contribute A_i ((eps+ + eps-) delta_ij/2 + (eps+ - eps-) n_i.G_j(c_i)) / area_f
 * instead (Eq. sheets), area_f being the body's total area.
 * n_i.G_i(c_i) is the principal value, 0 for a flat triangle.
 * A_dev: device, row-major double, (row1-row0) rows of leading dimension lda >= N+F.
 * precision: BEM_FP64 or BEM_MIXED (regular pairs rounded to FP32).
 */
int bem_assemble_rows(bem_ctx* ctx, int64_t row0, int64_t row1, int32_t precision, double* A_dev,
                      int64_t lda);

/*
 * y = A x without forming A (matrix-free): far pairs by the quadrature kernel,
 * near pairs from the precomputed closed-form values, then the row equations
 * above.  x_dev, y_dev: device double [nrhs][N+F].  1 <= nrhs <= 4.
 * precision: BEM_FP64, BEM_MIXED or BEM_DF.
 */
int bem_matvec(bem_ctx* ctx, int32_t precision, int32_t nrhs, const double* x_dev, double* y_dev);

/*
 * Right-hand side b of Eqs. Final1-Final4: b_i = V0 of row i's conductor, 0 on
 * every other row.  V0_dev: device double [nrhs][nregions] of conductor
 * potentials (entries of other regions ignored), or NULL for the mesh's V0.
 * b_dev: device double [nrhs][N+F].
 */
int bem_rhs(bem_ctx* ctx, int32_t nrhs, const double* V0_dev, double* b_dev);

/*
 * Solve A u = b (b from bem_rhs with V0_dev) by restarted GMRES with right
 * Jacobi scaling (Sec. 3; Sec. 5 names GMRES with a diagonal preconditioner) to
 * ||b - A u|| <= tol ||b|| (unpreconditioned 2-norm).  BEM_FP64: every matvec in
 * FP64.  BEM_MIXED: GMRES on the mixed matvec inside an iterative refinement
 * whose residual b - A u is formed with the FP64 matvec.  u_dev: device double
 * [nrhs][N+F]; its input value is ignored (start from 0).  iters (host, may be
 * NULL): total GMRES iterations; relres (host, may be NULL): final FP64 relative
 * residual per right-hand side, [nrhs].  Synchronises the stream (it reads the
 * Krylov coefficients back).  BEM_ERR_NOT_CONVERGED if tol was not reached within
 * max_iters (u then holds the last iterate).
 */
int bem_solve(bem_ctx* ctx, int32_t precision, int32_t nrhs, const double* V0_dev, double* u_dev,
              double tol, int32_t* iters, double* relres);

/*
 * phi and E at M arbitrary points (field formula of Sec. 2):
 *   phi(x) = sum_j u_j S_j(x),  E(x) = sum_j u_j G_j(x).
 * Points closer than eta R_j to a triangle's circumcentre take its closed form in
 * FP64.  A point lying exactly on a triangle gets the principal value of that
 * triangle's normal field.  u_dev: device double [>= N] (entries >= N ignored);
 * pts_dev: device double [M][3]; phi_dev: device double [M] or NULL; E_dev:
 * device double [M][3] or NULL.  Any M >= 0 (processed in chunks of max_points).
 */
int bem_eval_field(bem_ctx* ctx, int32_t precision, const double* u_dev, int64_t M,
                   const double* pts_dev, double* phi_dev, double* E_dev);

/*
 * Same result as bem_eval_field, for callers that cannot allocate device memory
 * when they evaluate the field (for example a process whose remaining GPU memory
 * belongs to its own arena after start-up, so that a further cudaMalloc fails or is
 * not allowed).  The paper has no counterpart; this is a property of the library.
 *
 * The call allocates nothing.  Its scratch (the far-field partial sums) is one fixed
 * 8 MiB array in the library's static device memory, which every GPU that loads the
 * library holds until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the context's device current;
 * make that first call before any stream capture.  The address is kept for the
 * life of the process: after cudaDeviceReset (or any teardown of the device's
 * primary context) it is stale, so do not call this entry point again after one.  All calls on a device share the
 * array, so calls whose GPU work overlaps (other streams, other threads, other
 * contexts on the same device) race and give wrong results: order them.  Nothing
 * needs clearing between calls (every partial read is written by the same call).
 * Limit: M <= 65536 points per call, else BEM_ERR_CAPACITY and no work is queued.
 * Arguments and layout as bem_eval_field; the context's device must be current.
 */
int bem_eval_field_static(bem_ctx* ctx, int32_t precision, const double* u_dev, int64_t M,
                          const double* pts_dev, double* phi_dev, double* E_dev);

/* Field-line tracing parameters (Eq. Breakdowncrit). */
typedef struct {
    double h;            /* RK4 step in arc length; default 1e-3 */
    double r_max;        /* stop where |x| = r_max; default 10 */
    double c, E0, d;     /* alpha_eff(E) = c (E - E0)^2 for E > E0, else -d; 1e-2, 0.5, 0.1 */
    double e_floor;      /* stop at a step start where |E| < e_floor; default 1e-12 */
    int64_t max_steps;   /* stop after this many steps; default 200000 */
} bem_trace_params;

void bem_default_trace_params(bem_trace_params* tp);

/*
 * Breakdown integral along field lines (Sec. 1, Eq. Breakdowncrit):
 *   K = int_gamma alpha_eff(|E|) ds,
 * gamma the field line through each seed, dx/ds = s0 E/|E|, s0 = sign(E.n) at the
 * seed (n: normal of the triangle whose centroid is nearest to the seed, so lines
 * leave the electrode), E the field of u (as bem_eval_field).  Classical RK4 with
 * step h on (x, K).  The branch of alpha_eff is part of the state; where a step
 * ends on the other side of |E| = E0 the crossing is located on the re-stepped RK4
 * step (Illinois regula falsi) and the step is split there, so K is a smooth
 * function of the data.  Stops, located the same way: |x| = r_max (status 1);
 * entering another conductor or floating body (status 2: the solid angle of its
 * triangles passes 2 pi).  At step starts: |E| < e_floor (status 4), non-finite
 * field (status -1: seed on an edge or vertex); max_steps steps: status 3.
 * u_dev: device double [>= N]; seeds_dev: device double [L][3]; tp: host, NULL =
 * defaults; outputs (device): K_dev double [L], status_dev int32 [L], nsteps_dev
 * int32 [L] (completed steps), xend_dev double [L][3] (end point), any may be NULL.
 * One persistent launch: a CTA of 8 warps traces up to 8 lines, one per warp, whose field
 * evaluations share the CTA's sweeps over the triangles; on meshes of 8,192 triangles
 * or more a thread-block cluster of up to 8 CTAs (params.trace_cluster, by default
 * chosen from the mesh size and L) shares each sweep, every CTA taking every
 * cluster-size-th group of 32 triangles (BEM_MIXED; contiguous parts in BEM_FP64);
 * the sums, grouped by those parts, then agree
 * between cluster sizes to rounding.  Precision BEM_FP64 or BEM_MIXED (regular pairs
 * in FP32).
 */
int bem_trace_lines(bem_ctx* ctx, int32_t precision, const double* u_dev, int64_t L,
                    const double* seeds_dev, const bem_trace_params* tp, double* K_dev,
                    int32_t* status_dev, int32_t* nsteps_dev, double* xend_dev);

/*
 * y = A^T x, the transpose of bem_matvec's operator (the adjoint solve needs it):
 * column j of A integrates over triangle j the potential of point charges (rows of
 * conductors and floating bodies) and dipoles along n_i (dielectric rows, and the
 * neutrality rows' weights) placed at the centroids.  x_dev, y_dev: device double
 * [N+F].  precision: BEM_FP64 or BEM_MIXED.  Uses the column-ordered copy of the near
 * pairs that bem_create builds with the adjoint workspace (params.adjoint_lines > 0;
 * else BEM_ERR_CAPACITY); allocates nothing.  far_order 2..4.
 */
int bem_matvec_transpose(bem_ctx* ctx, int32_t precision, const double* x_dev, double* y_dev);

/*
 * Gradient of J = sum_l w_l K_l (K_l = bem_trace_lines' breakdown integral of line
 * l, w_l = dL_dK_dev[l]) with respect to the vertex coordinates, the conductor
 * potentials and the permittivities, through the collocation system: for a design
 * objective built on Eq. Breakdowncrit (the paper's outlook names optimisation;
 * the adjoint itself is not in the paper).  u_dev must solve the system for the
 * mesh's V0 (bem_solve, same precision).  The discrete adjoint of what bem_solve
 * and bem_trace_lines compute: the lines are traced again keeping the state at the
 * start of every params.adjoint_checkpoint-th step; then, from the last segment to
 * the first, each segment's steps are traced once more from their checkpoint with a
 * record of every sub-step and reversed step by step (located crossings enter
 * through the implicit function theorem); the result does not depend on the
 * checkpoint interval.  A^T mu =
 * dJ/du is solved by GMRES, and -mu^T (dA/dtheta) u + mu^T db/dtheta is summed
 * pair by pair; regular pairs are differentiated on their quadrature nodes, near
 * pairs through the closed form with dual numbers.
 * Outputs (device, any may be NULL): K_dev double [L]; gX_dev double [nv][3];
 * gV0_dev double [nregions] (dJ/dV0 of every conductor region, 0 elsewhere);
 * geps_dev double [nregions][2] (dJ/d eps_plus, dJ/d eps_minus; eps_plus of a
 * floating region enters its neutrality row, and both permittivities of a sheet
 * enter its row of Eq. sheets).  Allocates nothing: it works in the adjoint workspace
 * of bem_create (params.adjoint_lines lines at a time, any L), and synchronises.
 * BEM_ERR_CAPACITY if the context has no adjoint workspace, or if tp->max_steps needs
 * more checkpoints per line than the workspace holds for even one line.  BEM_ERR_ARG
 * if a line ends on another electrode or in a singular field (status 2 or -1).
 * far_order 2..4.
 */
int bem_adjoint(bem_ctx* ctx, int32_t precision, const double* u_dev, int64_t L,
                const double* seeds_dev, const bem_trace_params* tp, const double* dL_dK_dev,
                double* K_dev, double* gX_dev, double* gV0_dev, double* geps_dev);

/*
 * Field on the + side of the surface at every centroid ("E surface" of Sec. 5):
 *   E+(c_i) = E_PV(c_i) + u_i n_i / 2   (Eq. ADL read as E+.n = sigma/2 + K' sigma).
 * E_dev: device double [N][3].
 */
int bem_surface_field(bem_ctx* ctx, int32_t precision, const double* u_dev, double* E_dev);

/*
 * Measured arithmetic peaks of the current CUDA device, the denominators of the
 * regular-pair kernels' roofline: fused multiply-add chains at full occupancy,
 * timed with CUDA events (best of three launches, about 0.1 s in all), 2 flops per
 * multiply-add.  fp32_tflops: the larger of the paired (fma on float2) and scalar
 * FP32 rates; fp32_scalar_tflops: the scalar rate; fp64_tflops: the FP64 rate.
 * Outputs are host pointers, any may be NULL.  Allocates and frees a small device
 * buffer and a private stream; synchronises.  Not part of the paper's method.
 * Errors: BEM_ERR_CUDA (message in bem_last_error(NULL)).
 */
int bem_measure_peaks(double* fp32_tflops, double* fp64_tflops, double* fp32_scalar_tflops);

/* ------------------------------------------------------------------ curved triangles
 * The paper's own discretisation (Sec. 3, Sec. 4): six-node triangles (corners, then
 * the midpoints of the edges 01, 12, 20, which may lie off the corners' plane: a
 * piecewise quadratic surface), the density sigma_h = sum_v u_v psi_v with psi_v the
 * mapped linear function that is 1 at vertex v, collocation at the vertices:
 *     v_ij = sum_T int psi_j(y) / (4 pi |x_i - y|) dS_y        (Eq. Matrix).
 * Pairs (vertex, triangle) are singular when the vertex is a corner of the
 * triangle (Duffy rule collapsed there, sing_order^2 points), regular when D > eta R
 * with the circumcircle of the corners (Duffy rule collapsed at corner 0, far_order^2
 * Gauss-Legendre points), near-singular otherwise (split at the point of the curved
 * triangle closest to the vertex, found by projected Gauss-Newton; each part a Duffy
 * rule collapsed there with near_radial points per geometric radial piece, refined
 * toward it down to a tenth of distance / size, and near_angular angular points).
 * Rows: conductor vertices sum_j v_ij u_j = V0 (Eq. Final1), floating vertices
 * sum_j v_ij u_j - V_f = 0 (Eq. Final2), one neutrality row per floating body in the
 * form Gauss's law gives a closed conductor, int_body sigma_h dS = 0 (Eq. Final4).
 * Dielectric and sheet regions are not built on this path.
 * The context this creates serves bem_destroy, bem_sizes, bem_get_counters,
 * bem_assemble_rows, bem_matvec (BEM_FP64, BEM_MIXED), bem_rhs, bem_solve (the
 * mixed form refines with the FP64 product) and bem_eval_field; the other calls
 * return BEM_ERR_ARG.  Unknowns: u at the vertices 0..nv-1, then V_f.
 */
typedef struct {
    double eta;              /* regular iff D > eta R; default 4 */
    int32_t far_order;       /* regular rule far_order x far_order points, 1..6; default 4 */
    int32_t sing_order;      /* singular rule sing_order x sing_order; default 24 */
    int32_t near_radial;     /* near-singular rule: points per radial piece; default 16 */
    int32_t near_angular;    /* near-singular rule: angular points; default 64 */
    int32_t gmres_restart, max_iters, max_refine;  /* as bem_params: 100, 2000, 6 */
    int32_t far32_variant;   /* packed FP32 kernel, 2, 3 or 4 target pairs per thread; default 2 */
    int64_t max_points;      /* as bem_params; default 131072 */
    int32_t timing;          /* as bem_params */
    int32_t reserved;
} bem_p1_params;

void bem_p1_default_params(bem_p1_params* p);

/*
 * Create a context of curved six-node triangles.  nodes: host double [nn][3], the
 * first nv of them the triangle corners (vertices, the collocation points); tri6:
 * host int32 [N][6] node indices (corners counter-clockwise about the outward
 * normal, then edge midpoints 01, 12, 20); region: host int32 [N]; regions: host
 * [nregions], conductor, floating or dielectric kinds (every vertex's triangles must
 * share its region).  A dielectric vertex's row is Eq. Final3 with K'u taken as the
 * mean of the two one-sided normal fields, each the field at x_i +- delta n_i
 * extrapolated to delta -> 0 from delta and 2 delta (delta = 1e-3 of the mean edge
 * length at the vertex, n_i the normalised sum of its triangles' normals there).
 * Set-up computes every singular and near-singular integral in FP64 on the device.  Errors: BEM_ERR_ARG, BEM_ERR_DEGENERATE (collinear corners),
 * BEM_ERR_NOMEM, BEM_ERR_CUDA; on error *out is NULL.
 */
int bem_p1_create(bem_ctx** out, int64_t nn, const double* nodes, int64_t nv, int64_t N, const int32_t* tri6,
                  const int32_t* region, int32_t nregions, const bem_region* regions,
                  const bem_p1_params* params, void* stream);

/* ------------------------------------------------------------------ batches
 * Many meshes (instances) of uneven size with up to four right-hand sides each,
 * served together: the operators are those of bem_matvec / bem_solve /
 * bem_trace_lines, only scheduled for a family of devices at once.
 *   - Regular pairs of all instances and right-hand sides run in ONE persistent
 *     launch whose CTAs take (instance, target tile, triangle slice) work items
 *     from an atomic counter; one pass over a pair's quadrature nodes serves all
 *     right-hand sides of its instance.
 *   - bem_batch_solve runs restarted GMRES(m) with right Jacobi scaling on all
 *     systems in lock step; a whole restart cycle (m Arnoldi iterations of all
 *     systems) is captured once as a CUDA graph and replayed once per cycle, with one
 *     host synchronisation (Hessenberg columns, rotations and stop tests on the
 *     device; iterations after every system has stopped do no work).
 *   - bem_batch_trace traces the lines of all instances in one persistent launch.
 * The batch owns its workspace (Krylov bases: (m+1) x (N_i+F_i) doubles per system)
 * and a private stream; every call orders itself after the work already queued on
 * the contexts' stream and makes that stream wait for its own work, so the calls
 * behave as if issued on the contexts' stream.  The contexts must stay alive and
 * unused by other calls while a batch call runs.
 */
typedef struct bem_batch bem_batch;

typedef struct {
    int64_t n_instances, nrhs;
    int64_t far_launches;     /* batched regular-pair launches (graph replays included) */
    int64_t pairs;            /* (target, triangle) pairs those launches covered */
    int64_t rhs_pairs;        /* pairs x right-hand sides */
    int64_t graph_launches;   /* replays of the restart-cycle graph (one per cycle) */
    int64_t kernel_launches;  /* kernels launched by the batch, graph nodes included */
    int64_t arnoldi_steps;    /* Arnoldi iterations summed over the systems */
    int64_t lines;            /* field lines traced */
    int64_t far_timed;        /* regular-pair launches timed (flags bit 0, bem_batch_matvec) */
    double far_ms;            /* their total time in milliseconds */
    int64_t eval_pairs;       /* (point, triangle) pairs of the batched field-point launches */
} bem_batch_counters;

/*
 * ctxs: host array of n >= 1 contexts on one device, created on one stream, with
 * the same far_order (2..4) and gmres_restart; nrhs: right-hand sides per instance,
 * 1..4 (system s = instance * nrhs + rhs).  flags bit 0: time the regular-pair
 * launch of bem_batch_matvec with CUDA events (synchronises).  GMRES limits
 * (max_iters, max_refine) and the residual form are those of ctxs[0].
 * BEM_ERR_ARG for mismatched contexts, BEM_ERR_NOMEM if the workspace does not fit.
 */
int bem_batch_create(bem_batch** out, bem_ctx* const* ctxs, int32_t n, int32_t nrhs, int32_t flags);
int bem_batch_destroy(bem_batch* b);
const char* bem_batch_last_error(const bem_batch* b);
int bem_batch_get_counters(bem_batch* b, bem_batch_counters* out);
int bem_batch_reset_counters(bem_batch* b);

/*
 * y_i = A_i x_i for every instance and right-hand side, with the mixed form's
 * products (FP32 regular pairs with compensated sums, FP64 near pairs; Eqs.
 * Final1-Final4).  x, y: host arrays of n device pointers, each to double
 * [nrhs][N_i+F_i].
 */
int bem_batch_matvec(bem_batch* b, const double* const* x, double* const* y);

/*
 * Solve A_i u_i = b_i(V0_i) for every instance and right-hand side (as bem_solve
 * with BEM_MIXED: GMRES on the FP32-regular-pair products inside an iterative
 * refinement whose residual uses the FP64-accurate operator) to |b - A u| <= tol |b|.
 * precision: BEM_MIXED only.  V0: host array of n device pointers to double
 * [nrhs][nregions_i] (conductor potentials per right-hand side), or NULL (the
 * regions' V0, nrhs = 1).  u: host array of n device pointers to double
 * [nrhs][N_i+F_i] (written).  iters, relres: host [n*nrhs] or NULL: Arnoldi
 * iterations and final relative residual per system.  Synchronises.
 * BEM_ERR_NOT_CONVERGED if a system missed tol (u holds the best iterate).
 */
int bem_batch_solve(bem_batch* b, int32_t precision, const double* const* V0, double* const* u,
                    double tol, int32_t* iters, double* relres);

/*
 * Field lines of every instance (as bem_trace_lines, without the end points).
 * u: host array of n device pointers to double [>= N_i]; L: host int64 [n] lines per
 * instance (0 allowed); seeds: host array of n device pointers to double [L_i][3];
 * K, status, nsteps: host arrays of n device pointers (each may be NULL, or the
 * array itself NULL).  One persistent launch; a CTA of 8 warps traces up to 8 lines at
 * a time, one per warp, taking lines of one mesh after another.
 * precision BEM_FP64 or BEM_MIXED.  Synchronises.
 */
int bem_batch_trace(bem_batch* b, int32_t precision, const double* const* u, const int64_t* L,
                    const double* const* seeds, const bem_trace_params* tp, double* const* K,
                    int32_t* const* status, int32_t* const* nsteps);

/*
 * phi and E at points of every instance (as bem_eval_field), for a family of meshes at
 * once.  BEM_MIXED: the regular pairs of all instances' points run in ONE persistent
 * launch per chunk of points (the chunk is the smallest params.max_points of the
 * contexts; work items of 256 points x a triangle slice common to all instances), in
 * each context's own far workspace; then each instance's FP64 near pass.  BEM_FP64:
 * each instance's bem_eval_field in turn.  u: host array of n device pointers to double
 * [>= N_i]; M: host int64 [n] points per instance (0 allowed); pts: host array of n
 * device pointers to double [M_i][3]; phi, E: host arrays of n device pointers to
 * double [M_i] and [M_i][3] (entries, or the arrays, may be NULL).  Allocates nothing;
 * asynchronous like bem_eval_field.  The paper evaluates one device at a time; this
 * call serves the batch.
 */
int bem_batch_eval_field(bem_batch* b, int32_t precision, const double* const* u, const int64_t* M,
                         const double* const* pts, double* const* phi, double* const* E);

#ifdef __cplusplus
}
#endif

#endif /* BEM_H */
