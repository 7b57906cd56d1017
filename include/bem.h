/*
 * bem.h — C ABI of the GB300 FMM-accelerated boundary-element library (libbem.so).
 *
 * The library computes the collocation boundary-element operators of the bubble-dynamics
 * method of Gumerov, Pityuk, Abramova and Akhatov (arXiv:1905.01341):
 *   - single layer  L[q](r_i)   ~ sum_j L_ij q_j,    double layer M[phi](r_i) ~ sum_j M_ij phi_j
 *     (Section 3.1, Eq. (d1)), kernels G = 1/(4 pi |r - r'|) and dG/dn' = n'.(r - r')/(4 pi |r - r'|^3)
 *     with the normal pointing out of the bubble (Eq. (2.13));
 *   - off-diagonal entries by the one-point vertex quadrature L_ij = s_j G(r_i, r_j),
 *     M_ij = s_j dG/dn_j(r_i, r_j), i != j, with s_j = (1/3) sum A_k and n_j the normalised
 *     area-weighted triangle normal (Section 3.2, Eq. (ns1));
 *   - singular diagonals from the integral identities M_ii = -1/2 - sum_{j!=i} M_ij (Eq. (s3))
 *     and L_ii = n_i . [sum_{j!=i} (M_ij r_j - L_ij n_j) + (1/2 + M_ii) r_i] (Eq. (s5));
 *   - the combined product (f L + g M) X (Eq. (3.27)) by the fast multipole method
 *     (Section 3.7: octree to uniform depth, multipole/local expansions truncated at degree
 *     p_fmm - 1) or by the direct O(N^2) sum (Section 3.9, "GPU" brute force);
 *   - the Dirichlet solve L q = b, b = -phi/2 + M phi (Eqs. (3.1)-(3.2)) by GMRES started from
 *     a caller-given guess (Section 3.8): unpreconditioned as in the paper, or right-
 *     preconditioned (bem_params.gmres_precond); every variant stops on the same true residual.
 *
 * Conventions (all entry points):
 *   - Every function returns a bem_status (0 = BEM_OK). No C++ exception crosses the ABI.
 *     On failure bem_last_error(ctx) returns a NUL-terminated message owned by the context,
 *     valid until the next call on that context.
 *   - Array arguments are plain pointers. Each may point to host memory or to device
 *     memory of the context's device; the library detects which. Device arrays are read and
 *     written in order on the context's stream; host arrays are copied through internal
 *     device buffers and the call returns after the host output is written.
 *   - The caller owns every array it passes; the library never keeps a caller pointer
 *     beyond the call. The context owns all internal buffers.
 *   - Vertex arrays are indexed in the caller's vertex order. Coordinates are SoA:
 *     xyz[0..N) = x, xyz[N..2N) = y, xyz[2N..3N) = z (double). Triangles are SoA int32:
 *     tri[0..T) = first corner, tri[T..2T) = second, tri[2T..3T) = third; corners are
 *     counter-clockwise seen from the liquid (outward normal, Section 3.4).
 *   - The API is FP64. The precision mode changes internal arithmetic only.
 *   - A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef BEM_H_
#define BEM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BEM_OK = 0,
    BEM_ERR_ARG = 1,       /* invalid argument (null pointer, size, parameter range)          */
    BEM_ERR_MESH = 2,      /* invalid mesh (index out of range, isolated vertex, zero normal) */
    BEM_ERR_NOT_BUILT = 3, /* apply/solve before bem_mesh_upload + fmm_build                  */
    BEM_ERR_NOCONV = 4,    /* GMRES hit maxit; q holds the last iterate, relres is set        */
    BEM_ERR_TIMEOUT = 5,   /* a bounded device wait ran out                                   */
    BEM_ERR_CUDA = 6,      /* CUDA runtime error                                              */
    BEM_ERR_NAN = 7,       /* non-finite vertex coordinate (fmm_build) or value in a result   */
    BEM_ERR_NOMEM = 8      /* device allocation failed                                        */
} bem_status;

typedef enum {
    BEM_PREC_FP64 = 0,  /* every kernel in FP64                                                */
    BEM_PREC_MIXED = 1  /* near field and expansions in FP32 with compensated sums; geometry,
                           diagonal assembly, GMRES and all API vectors stay FP64            */
} bem_precision;

typedef enum {
    BEM_MVP_FMM = 0,    /* fast multipole method (Section 3.7)                                */
    BEM_MVP_DIRECT = 1  /* direct all-pairs sum (Section 3.9 brute force; small N)            */
} bem_mvp_kind;

/* Parameters of a context. Fill with bem_params_default() and override fields. */
typedef struct {
    int32_t p_fmm;          /* truncation number: degrees 0..p_fmm-1, p_fmm^2 coefficients
                               per expansion (Section 3.7). Range 2..20. Default 14.           */
    int32_t leaf_target;    /* target mean points per non-empty leaf box (the clustering
                               parameter s of Section 3.6); 0 = autotune: the first build after
                               a mesh upload times single-layer products at the depth for 64
                               points per leaf and one level either side, and at that depth the
                               tensor-core M2L's pipeline depth and the near field's grid
                               (m2l_stages, p2p_blocks_per_sm where set to automatic), and keeps
                               the fastest combination for this mesh. Default 64.             */
    int32_t fixed_level;    /* > 0: force the octree depth l_max to this value (2..10).        */
    int32_t precision;      /* bem_precision. Default BEM_PREC_MIXED.                          */
    int32_t mvp;            /* bem_mvp_kind. Default BEM_MVP_FMM.                              */
    int32_t diag_precision; /* precision of the 4-RHS product that feeds Eqs. (s3)/(s5);
                               -1 = same as `precision`. Default -1.                           */
    int32_t diag_p_fmm;     /* truncation number of that 4-RHS product (2..20); -1 = p_fmm + 2,
                               at most 20. The identities form L_ii and M_ii by cancelling
                               O(1) sums down to O(h), which magnifies the far field's
                               truncation error; the products of GMRES do not need it (on the
                               3.21M-unknown cluster at p_fmm = 14 the off-diagonal part of a
                               product is within 6e-7 of the direct sum, L_ii within 4e-5).
                               Default -1.                                                     */
    int32_t overlap;        /* within a product, the near field runs on its own stream,
                               concurrently with the far field: 1 = from the start of the far
                               field, 2 = from the start of the M2L (the P2M runs alone, then
                               the near field fills the SMs around the tensor-core M2L);
                               0 = one stream, phase after phase (the per-kernel timings of a
                               profile then do not overlap); -1 = automatic (the tile
                               autotuner's choice between 1 and 2 when leaf_target = 0, else
                               1). Same results in every mode. Default -1.                     */
    int32_t m2l_tensor_cores; /* Mixed precision only. 1: single-RHS products (every GMRES
                               product) run M2L on the tensor cores (three-piece BF16 split,
                               FP32 accumulation) when p^2 is a multiple of 4 and <= 256;
                               2: the 4-RHS product behind the diagonals (Eqs. (s3)/(s5)) as
                               well, at diag_p_fmm; 3: as 2 while every bubble has at most
                               2562 vertices, else as 1 (the identities magnify the far
                               field's rounding by about R/h); 0: FP32 CUDA cores throughout.
                               Orders with p^2 > 256 use the CUDA cores in every mode.
                               Default 3.                                                      */
    int32_t gmres_precond;  /* 0: unpreconditioned GMRES, as in the paper (Section 3.8);
                               1: right Jacobi preconditioning x = D^-1 y with D = diag(L_ii)
                               (removes the spread of the single layer's scale across bubbles
                               of different radii);
                               2: right bubble-block preconditioning: per distinct bubble mesh
                               (same connectivity), the inverse of the isolated representative
                               bubble's single-layer block (built from the geometry of the
                               first solve after a mesh upload and kept), scaled by each
                               bubble's current size; removes the spread of each bubble's own
                               spectrum (R/(2n+1) on a sphere). Needs bubbles; memory n^2
                               doubles + n^2 floats per distinct mesh of n vertices.
                               Every mode stops on the same true residual |b - L q| / |b|.
                               Default 0.                                                      */
    int32_t gmres_maxit;    /* maximum GMRES iterations. Default 100.                          */
    int32_t gmres_restart;  /* restart length; 0 = no restart (= maxit). Default 0.            */
    double gmres_tol;       /* stop when |b - L q| / |b| <= tol (Section 3.8). Default 1e-6.  */
    int32_t m2l_stages;     /* shared-memory pipeline stages of the pair-major tensor-core M2L
                               (m2l_target_major = 0; the target-major kernel uses 3): 2 or 3;
                               0 = automatic (the tile autotuner's choice when leaf_target = 0,
                               else 3). Fewer stages leave shared memory on each SM for the
                               near field running concurrently. Default 0.                    */
    int32_t p2p_blocks_per_sm; /* near-field grid: 0 = one warp per work unit (all units in one
                               grid); k > 0 = a persistent grid of k blocks per SM looping over
                               the units, which leaves room on every SM for the far-field
                               kernels of the concurrent stream. Same results either way.
                               -1 = automatic (the tile autotuner's choice when leaf_target = 0,
                               else 0). Default -1.                                           */
    int32_t m2l_order_margin; /* truncation of each M2L translation by the separation of its
                               offset class (Section 3.7 truncates every translation at p_fmm):
                               -1 = every class at p_fmm; k >= 0 = class c at
                               p_c = min(p_fmm, ceil(p_fmm ln(rho_0) / ln(rho_c)) + k), where
                               rho_c = a / (|d_c| - a) is the convergence ratio of the
                               multipole-to-local series for boxes whose centres are |d_c| box
                               sizes apart (a = sqrt(3)/2, the box's circumradius) and rho_0 that
                               of the nearest class (d = (2, 0, 0)): every class is truncated
                               where its error bound falls to the nearest class's bound at p_fmm,
                               k degrees further. Measured against the direct sum, k = 6 keeps
                               the product error within ~5 % of the untruncated one at p_fmm 14
                               (mixed) and within 2x at 16 (FP64), for about 38 % of the M2L
                               multiply work. Default 6.                                      */
    int32_t m2l_target_major; /* layout of the tensor-core M2L (mixed precision): 1 = target-major
                               (per tile of target boxes, the MMAs of a few offset classes
                               accumulate in tensor memory; no row per translation); 0 =
                               pair-major (one product row per translation, summed per target
                               afterwards). Both sum in a fixed order. Default 1.             */
} bem_params;

/* Run-time counters of a context (cumulative since bem_create or bem_reset_stats). */
typedef struct {
    int64_t n_apply;        /* operator products (each multi-RHS product counts once)          */
    int64_t n_apply_rhs;    /* right-hand sides processed by those products                    */
    int64_t p2p_pairs;      /* near-field (or direct) source-receiver pairs per RHS, last build */
    int64_t m2l_pairs;      /* M2L translations per RHS, all levels, last build               */
    int32_t levels;         /* octree depth l_max of the last build                            */
    int32_t leaves;         /* non-empty leaf boxes of the last build                          */
    int32_t last_iters;     /* GMRES iterations of the last solve                              */
    int32_t last_mvps;      /* operator products of the last solve (iterations + 2)            */
    double last_relres;     /* true relative residual of the last solve                        */
    double last_build_ms;   /* device time of the last fmm_build                               */
    int64_t n_launches;     /* kernels launched by the library in this process (all contexts)   */
    int32_t m2l_stages;     /* tensor-core M2L pipeline stages in use (0 = the default, 3)      */
    int32_t overlap;        /* near-field / far-field overlap mode in use (bem_params.overlap)  */
    int32_t reserved;
    int32_t p2p_blocks_per_sm; /* near-field grid in use (0 = one warp per work unit)           */
    int64_t m2l_macs;       /* multiply-adds of one RHS's M2L, last build: sum over the pairs of
                               (truncated size)^2, the size padded to a multiple of 16 (the
                               tensor-core tiles): p_c^2 rounded up; = pairs x P^2 untruncated */
} bem_stats;

/* Phases reported by bem_profile_read, in this order. */
#define BEM_NUM_PHASES 15
/* geometry, tree, operators, strengths, p2m, m2m, m2l (tensor-core translations and the split
 * of the multipoles), l2l, l2p, p2p, direct, diag, gmres, m2l_reduce (per-target sums of the
 * M2L products), m2l_cc (M2L translations on the CUDA cores) */

/* Fill *p with the defaults listed above. */
int bem_params_default(bem_params *p);

/* Create a context on the current CUDA device. `stream` is a cudaStream_t (NULL = the
 * legacy default stream); every kernel of the context runs on it. */
int bem_create(void **ctx_out, const bem_params *p, void *stream);

/* Destroy a context and free its device memory. Accepts NULL. */
void bem_destroy(void *ctx);

/* Change the stream of an existing context. */
int bem_set_stream(void *ctx, void *stream);

/* Message of the last failed call on ctx (or, when ctx is NULL, of the last failed call on
 * this host thread that takes no context: bem_create, bem_apply_direct_noalloc). */
const char *bem_last_error(const void *ctx);

/* Section 2.1/3.1: upload the surface mesh. N vertices (collocation points) with SoA
 * coordinates xyz[3N]; T triangles tri[3T] (SoA, 0-based vertex indices); M bubbles with
 * vert_off[M+1] and tri_off[M+1] (bubble m owns vertices vert_off[m]..vert_off[m+1]-1 and
 * triangles tri_off[m]..tri_off[m+1]-1). Copies the data into the context and invalidates
 * any previous build. Returns BEM_ERR_ARG for bad sizes or offsets. */
int bem_mesh_upload(void *ctx, int64_t N, const double *xyz, int64_t T, const int32_t *tri,
                    int64_t M, const int64_t *vert_off, const int64_t *tri_off);

/* Independent clusters stepped together (one launch per phase for all of them): after
 * bem_mesh_upload, group the bubbles into C clusters, cluster c owning bubbles
 * bubble_off[c]..bubble_off[c+1]-1 (bubble_off[C+1]: 0 .. M, every cluster non-empty,
 * C <= 256). Each cluster gets its own octree cube (the cluster id sits in the high bits of
 * the Morton key, depth <= 8 per cluster), no interaction crosses clusters, and the singular
 * diagonals use each cluster's own sums; the products and solves therefore equal those of the
 * clusters taken one by one. Invalidates the build; a new bem_mesh_upload resets to one
 * cluster. */
int bem_mesh_set_clusters(void *ctx, int64_t C, const int64_t *bubble_off);

/* After a solve of a clustered mesh (bem_mesh_set_clusters with C > 1), per cluster: the GMRES
 * iterations it took, its true relative residual |b_c - L_c q_c| / |b_c|, and the device ms from
 * the start of that solve until its solution was final; *solve_ms gets the solve's device ms.
 * Clustered solves run one GMRES per cluster in lockstep (Section 3.8 for each cluster's own
 * system): one operator product per iteration serves all clusters, and each cluster stops and
 * takes its solution at the iteration where its own residual meets gmres_tol (a single
 * Krylov space over all clusters would stop on the global residual). Any array may be NULL. */
int bem_get_cluster_stats(void *ctx, int64_t C, int32_t *iters, double *relres, double *done_ms, double *solve_ms);

/* Section 3.9 (Table 1): upload N free points (SoA xyz[3N]) instead of a mesh, for the FMM's
 * accuracy study with monopoles. Weights are 1 and there is no singular diagonal, so after
 * fmm_build, bem_apply(ctx, 1, q, 0, NULL, out) gives out_i = sum_{j != i} q_j / (4 pi |r_i - r_j|). */
int bem_points_upload(void *ctx, int64_t N, const double *xyz);

/* Replace the vertex coordinates of the uploaded mesh (same N, same triangles), as a
 * time step does (Eq. (3.14)); invalidates the build. */
int bem_mesh_update_xyz(void *ctx, const double *xyz);

/* Section 3.2 and 3.7: vertex weights and normals (Eq. (ns1)), the octree (bounding cube,
 * Morton keys, radix sort, level boxes, neighbour and M2L lists), the FMM translation
 * operators, and the singular diagonals (Eqs. (s3), (s5)) from one 4-RHS product.
 * Returns BEM_ERR_NAN for a non-finite vertex coordinate (checked first) or diagonal, and
 * BEM_ERR_MESH for an isolated vertex or a zero area-weighted normal. */
int fmm_build(void *ctx);

/* Eq. (3.27): out = f L xL + g M xM (diagonals included). xL may be NULL when f == 0 and
 * xM may be NULL when g == 0. All vectors have length N. */
int bem_apply(void *ctx, double f, const double *xL, double g, const double *xM, double *out);

/* Eq. (d1): out = L q (single layer, with L_ii). */
int bem_apply_sl(void *ctx, const double *q, double *out);

/* Eq. (d1): out = M phi (double layer, with M_ii; no -phi/2 term). */
int bem_apply_dl(void *ctx, const double *phi, double *out);

/* Eq. (3.1): b = -phi/2 + M phi. */
int bem_rhs(void *ctx, const double *phi, double *b);

/* Eqs. (3.1)-(3.2), Section 3.8: given phi on S solve L q = b by GMRES with initial guess
 * q_inout (in), returning q in q_inout. iters and relres may be NULL. relres is the relative
 * residual |b - L q| / |b| evaluated with operator products, not GMRES's estimate: b - L q_0 for
 * the initial guess, then r_0 - L d at the end of every restart cycle (d the cycle's update of q),
 * and the solve stops when it meets gmres_tol. Returns BEM_ERR_NOCONV when maxit is reached. */
int bem_solve(void *ctx, const double *phi, double *q_inout, int32_t *iters, double *relres);

/* The bubble-block preconditioner of the solve with gmres_precond = 2, applied once:
 * z = P y with P = blockdiag_m (1 / R_m) Inv_k(m), Inv_k the inverse of the isolated
 * single-layer block (Eq. (d1), its diagonal from the identity of Eq. (s5) summed over that
 * bubble alone) of the first bubble with mesh connectivity k, scaled to unit size, and R_m the
 * current mean centroid distance of bubble m. Built on the first use after a mesh upload from
 * the geometry of that moment; the scales follow the current geometry. y and z have length N
 * (caller's vertex order, host or device memory, not overlapping). Mixed precision: one
 * tensor-core product per connectivity class, operands split into three BF16 pieces and
 * accumulated in FP32 (FP32 accuracy); FP64: an FP64 product. Returns BEM_ERR_ARG without
 * bubble offsets, BEM_ERR_MESH for a non-positive pivot in the setup, BEM_ERR_TIMEOUT when a
 * tensor-core wait ran out (the output is then undefined). */
int bem_precond_apply(void *ctx, const double *y, double *z);

/* Copies of the geometry of the last build, in the caller's vertex order: s[N], n[3N]
 * (SoA), Ldiag[N], Mdiag[N]. Any pointer may be NULL. */
int bem_get_geometry(void *ctx, double *s, double *n, double *ldiag, double *mdiag);

/* ------------------------------------------------------------------------------------------
 * Time step (Sections 3.4-3.6): dr/dt = n q, dphi/dt = (alpha v_t + v/2).v - (p_g - 2 sigma H)
 * + F(t) with alpha = -1 (Eqs. (3.13)-(3.15), g = 0), tangential velocity from Stokes' theorem
 * (Eqs. (3.7)-(3.11)), mean curvature from a paraboloid through five neighbours
 * (Eqs. (parab1)-(parab2)), polytropic gas (Eq. (2.8)), spherical shape filter on the inputs
 * and outputs of every right-hand-side evaluation (Eqs. (3.22)-(3.25)), 6th-order
 * Adams-Bashforth started by 4th-order Runge-Kutta (Section 3.5) by default; the other schemes
 * Section 3.5 names (Adams-Bashforth of orders 1-6, Adams-Bashforth-Moulton of orders 4-6,
 * Runge-Kutta starts of orders 4-6) are selected in bem_step_params.
 * Dimensionless units: lengths by a0, pressure by p0, time by a0 (rho/p0)^(1/2); rho = p0 = 1.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    double sigma;    /* surface tension sigma/(p0 a0). Default 0.073 (water, a0 = 10 um)        */
    double kappa;    /* polytropic exponent of Eq. (2.8). Default 1.4                           */
    double pa;       /* acoustic amplitude Pa/p0; p_inf = 1 - pa sin(omega t) (Eq. (2.6)). 1.0 */
    double omega;    /* angular frequency in units of (p0/rho)^(1/2)/a0. Default 1.2566 (200 kHz,
                        a0 = 10 um)                                                            */
    double courant;  /* C of Eq. (3.12): dt = C min(edge length at t = 0) / pa^(1/2). Default 0.1 */
    double dt;       /* > 0: fixed step used instead of the Courant rule. Default 0              */
    int32_t pf;      /* shape-filter bandwidth p_f: degrees 0..p_f-1. 0 = no filter. Default 6  */
    int32_t guess;   /* initial guess of each Adams-Bashforth step's solve: 0 = the q of the
                        previous solve (the paper, Sections 3.5, 3.8); k = 1, 2 or 3 = the
                        polynomial of degree k in t through the solutions at the last k + 1
                        step starts, evaluated at the new step's time. Runge-Kutta steps
                        always start from the previous solve (their k4 solve is at the new
                        step's time). Only the starting point of GMRES changes: every solve
                        still runs to gmres_tol. Not used while the learned guess is active.
                        Default 2 (degree 3 extrapolates the solves' rounding further).       */
    int32_t ab_order;  /* order k of the Adams-Bashforth steps, 1..6 (Section 3.5). Default 6    */
    int32_t corrector; /* 1: Adams-Moulton corrector of order k after each Adams-Bashforth
                          prediction (a predictor-corrector, two right-hand sides per step; k in
                          4..6). Default 0                                                    */
    int32_t rk_order;  /* order of the Runge-Kutta steps that start the integration until k - 1
                          past right-hand sides exist: 4 (classical), 5 (Butcher's six-stage) or
                          6 (Butcher's seven-stage). Default 4                                 */
} bem_step_params;

typedef struct {
    double t;              /* time after the step                                              */
    double dt;             /* step size                                                        */
    int32_t rhs_calls;     /* right-hand-side evaluations in the step (4/6/7 for an RK4/5/6 start
                              step, 1 for Adams-Bashforth, 2 with the corrector)              */
    int32_t gmres_iters;   /* GMRES iterations summed over those evaluations                  */
    int32_t mvps;          /* operator products, counting each 4-RHS diagonal product once    */
    int32_t nonconverged;  /* solves that stopped at maxit (the step still advances)          */
    double max_relres;     /* largest final relative residual among the step's solves         */
    int64_t steps;         /* steps taken since bem_step_init                                 */
} bem_step_stats;

/* Fill *sp with the defaults listed above. */
int bem_step_params_default(bem_step_params *sp);

/* Start a time integration from the uploaded mesh (r at t = 0), phi0[N] and an optional
 * initial guess q0[N] for the first GMRES solve (NULL = zeros). Builds one shape
 * filter per distinct initial bubble shape (bubbles whose unit directions from their centroid
 * coincide share it): the spherical filter (real spherical harmonics of degrees 0..p_f-1) for a
 * sphere-like bubble (Euler characteristic V - T/2 = 2), the toroidal filter (real 2D Fourier
 * basis of the torus angles, |n|, |m| <= p_f/2, Eq. (spherical7)) for a ring-like one (0); the
 * torus axis is the direction of least second moment of the bubble's initial vertices about its
 * centroid. Also the five-neighbour lists of the curvature fit, V_m0 and a_m0, and the step
 * size. Returns BEM_ERR_MESH when a bubble is neither sphere- nor ring-like, its filter is
 * singular, or a vertex has fewer than five neighbours. */
int bem_step_init(void *ctx, const double *phi0, const double *q0, const bem_step_params *sp);

/* Advance one step; st may be NULL. */
int bem_step(void *ctx, bem_step_stats *st);

/* Current state: xyz[3N] (SoA), phi[N], the last q[N] and t. Any pointer may be NULL. */
int bem_step_get_state(void *ctx, double *xyz, double *phi, double *q, double *t);

/* Eqs. (3.22)-(3.25): the shape filter of the time integration applied once, y = x^ with
 * x^ = G (G+ x) per bubble for each of the four fields of x = (xyz [3N] SoA, phi [N]), using the
 * bases that bem_step_init built (spherical harmonics of degree < pf, or the torus basis for a
 * ring-shaped bubble; the identity when pf = 0). Mixed precision evaluates it in compensated
 * FP32 (G and G+ as (hi, lo) pairs, about 48 bits), FP64 in FP64. x and y have length 4N, host
 * or device memory, and may be the same array. Returns BEM_ERR_NOT_BUILT before bem_step_init. */
int bem_step_filter(void *ctx, const double *x, double *y);

/* Replace the current state: xyz[3N] (SoA), phi[N] and the q[N] the next solve starts from (or
 * extrapolates with); any pointer may be NULL (that part is kept). The time, the step size and
 * the history of right-hand sides (Section 3.5) are kept, so the next bem_step continues the
 * integration from the given state: a caller that holds the state in its own (host) memory
 * passes it back each step. */
int bem_step_set_state(void *ctx, const double *xyz, const double *phi, const double *q);

/* Checkpoint and resume of a time integration (the paper has none; Sections 3.5-3.6 define
 * what a step depends on). A checkpoint holds what evolves: r and phi, the last q, t, dt, the
 * step count, the right-hand sides of the last five step starts (the Adams-Bashforth history,
 * Section 3.5) and the step-start solutions behind the extrapolated initial guess; and what
 * the fixed parts are rebuilt from: r at t = 0, the step parameters and the tuned octree depth.
 * It is a byte buffer of *size bytes (host or device memory of the context's device): call
 * bem_step_save with buf = NULL to get the size, then with a buffer of at least that many
 * bytes (cap). Learned-guess weights are saved separately (bem_mlp_get_params).
 * bem_step_load needs a context holding the same mesh connectivity (N, T, M and offsets as
 * uploaded; coordinates are replaced): it rebuilds the shape filters, V_m0, a_m0, neighbour
 * lists and step size from r(0) as bem_step_init does, restores the evolving state, and the
 * next bem_step continues the saved run. With identical context parameters, a fixed octree
 * depth (fixed_level, or a saved tuned depth) and gmres_precond 0 or 1, the continued run
 * repeats the original bit for bit on the same GPU; the bubble-block preconditioner
 * (gmres_precond 2) is rebuilt from the geometry at the first solve after the load, so those
 * solves start differently and agree with the original within the GMRES tolerance. Returns
 * BEM_ERR_ARG for a buffer that is too small, not a checkpoint, or of another mesh size. */
int bem_step_save(void *ctx, void *buf, int64_t cap, int64_t *size);
int bem_step_load(void *ctx, const void *buf, int64_t size);

/* ------------------------------------------------------------------------------------------
 * Learned GMRES initial guess. The paper starts each solve from the previous step's q
 * (Sections 3.5, 3.8); that, or its extrapolation in t (bem_step_params.guess), is the base
 * start and the fallback. Per bubble, the features are the least-squares real
 * spherical-harmonic coefficients (degree <= lmax, on the bubble's initial directions, as in
 * the shape filter, Eqs. (3.22)-(3.23)) of phi, of the base start q_b, and of q_b minus the base
 * start of the solve before; a multilayer perceptron (3 hidden relu layers) predicts the
 * correction of q's coefficients, c(q) - c(q_b), and the guess is q_b + G y. Features and
 * targets are scaled per column by their root mean square over the recorded samples, computed
 * when bem_mlp_train is called (those scales are not part of the parameter vector). Samples are
 * recorded and the guess is used in the Adams-Bashforth phase of bem_step (one solve per step).
 * Products run on the tensor cores in BF16 with FP32 accumulation; weights keep an FP32 master
 * copy; training is Adam on the mean squared error.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t dims[5];          /* layer widths: 3 (lmax+1)^2, hidden, hidden, hidden, (lmax+1)^2 */
    int32_t reserved;
    int64_t num_params;       /* weights and biases: W1, b1, ..., W4, b4 (W row-major [out][in]) */
    int64_t samples;          /* recorded (features, target) rows, one per bubble per solve      */
    int64_t compared_solves;  /* solves run from both starts (compare mode)                      */
    int64_t iters_guess;      /* their GMRES iterations from the learned guess                    */
    int64_t iters_fallback;   /* ... and from the base start q_b                                  */
    double res0_guess;        /* summed initial relative residuals from the learned guess         */
    double res0_fallback;     /* ... and from the base start q_b                                  */
} bem_mlp_summary;

/* Create the network (He initialisation from `seed`, output layer scaled by 0.1) after
 * bem_step_init. hidden: multiple of 16 in 16..256; lmax in 0..10. The features use spherical
 * harmonics: BEM_ERR_MESH when a bubble is not sphere-like. */
int bem_mlp_init(void *ctx, int32_t hidden, int32_t lmax, uint64_t seed);

/* record: store (features, c(q) - c(q_b)) of every bubble at every solve of bem_step;
 * use_guess: start every solve from the learned guess; compare: with use_guess, also solve from
 * the base start q_b (the result of that solve is discarded) and accumulate both iteration
 * counts. */
int bem_mlp_set_mode(void *ctx, int32_t record, int32_t use_guess, int32_t compare);

/* Adam (lr, beta = 0.9/0.999) over the recorded rows, in minibatches of `batch` rows, for
 * `epochs` passes; *last_loss = mean loss of the last pass. */
int bem_mlp_train(void *ctx, int32_t epochs, int32_t batch, double lr, double *last_loss);

/* Loss and gradients for one batch: F[B][dims[0]], T[B][dims[4]] -> *loss,
 * grads[num_params] in parameter order. */
int bem_mlp_loss_grad(void *ctx, int32_t B, const double *F, const double *T, double *loss, double *grads);

/* Network output Y[B][dims[4]] for features F[B][dims[0]]. */
int bem_mlp_forward(void *ctx, int32_t B, const double *F, double *Y);

/* Parameters as one FP64 vector of num_params entries, in parameter order. */
int bem_mlp_get_params(void *ctx, double *out);
int bem_mlp_set_params(void *ctx, const double *in);

/* Sizes, sample count and compare-mode counters. */
int bem_mlp_info(void *ctx, bem_mlp_summary *out);

/* Allocation-free direct product. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory at the time of the call, such as code running
 * inside another framework's fixed memory pool or a latency-critical loop where a device
 * allocation (which synchronises the device) is not acceptable.
 * Computes out = f L xL + g M xM (diagonals included) by the direct all-pairs sum with the
 * FP32 kernel of BEM_PREC_MIXED + BEM_MVP_DIRECT, the same result as bem_apply on a context
 * with those parameters. Takes no context: xyz[3N] (SoA), s[N], n[3N] (SoA), ldiag[N],
 * mdiag[N] (for example from bem_get_geometry), xL[N], xM[N] and out[N] are device memory
 * of the current device; the caller owns them. Runs on `stream` (a cudaStream_t; NULL = the
 * legacy default stream) and returns without waiting for the result.
 * It allocates nothing: its only scratch, the hi + lo FP32 split of the coordinates, lives in
 * a file-scope device array sized for N <= 262144 (6 MiB, held by every GPU that loads the
 * library until the process exits). N outside 2..262144 returns BEM_ERR_ARG with a message in
 * bem_last_error(NULL). Every array must be device memory of the current device (or managed
 * memory); a host or unregistered pointer returns BEM_ERR_ARG before anything is launched (the
 * library cannot check lengths: the caller guarantees them). The first call on a device looks
 * up that array's device address, with that device current (safe from several host threads);
 * make this first call before any stream capture. The address is cached for the process, so do
 * not call this entry point on a device after cudaDeviceReset. Every call shares the array and
 * overwrites it, so calls that overlap on the GPU (different streams, or different host
 * threads) race. */
int bem_apply_direct_noalloc(int64_t N, const double *xyz, const double *s, const double *n, const double *ldiag,
                             const double *mdiag, double f, const double *xL, double g, const double *xM,
                             double *out, void *stream);

/* Residual history of the last bem_solve: the true relative residual at the start of each
 * GMRES cycle and the estimate |g_{k+1}|/|b| after each iteration, in order; the final entry
 * is the true relative residual of the returned q. Writes up to `max` values to out and the
 * total count to *count. */
int bem_get_residual_history(void *ctx, double *out, int32_t max, int32_t *count);

/* The truncation order p_c of each of the 316 M2L offset classes for expansion order p_fmm and
 * margin (bem_params.m2l_order_margin; -1 = p_fmm for all). Classes are the offsets
 * (x, y, z) in [-3, 3]^3 with max(|x|, |y|, |z|) >= 2 of the source box from the target box in
 * units of the box size, in lexicographic order (x slowest). Needs no GPU. */
int bem_m2l_orders(int32_t p_fmm, int32_t margin, int32_t *orders);

/* Counters; see bem_stats. */
int bem_get_stats(void *ctx, bem_stats *out);
int bem_reset_stats(void *ctx);

/* Per-phase device timing. While enabled, each phase's kernels are bracketed by CUDA events
 * recorded on the context's stream (a few microseconds of overhead per phase). */
int bem_profile_enable(void *ctx, int on);

/* Synchronises the context's stream and returns, per phase (BEM_NUM_PHASES entries), the
 * device milliseconds and the number of timed intervals recorded since the last read; then
 * clears the records. Either array may be NULL. */
int bem_profile_read(void *ctx, double *ms, int64_t *intervals);

/* Name of phase i (0 <= i < BEM_NUM_PHASES), or NULL. */
const char *bem_phase_name(int i);

#ifdef __cplusplus
}
#endif

#endif /* BEM_H_ */
