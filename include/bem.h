/*
 * libbem -- FMM-accelerated boundary-element solver for continuum (Poisson)
 * biomolecular electrostatics on one GB300 GPU (sm_103a).
 *
 * Method: Yokota, Bardhan, Knepley, Barba, Hamada, "Biomolecular
 * electrostatics using a fast multipole BEM on up to 512 GPUs and a billion
 * unknowns" (arXiv:1007.4591).  Section references below are to that paper.
 *
 * Model (Sec. 2.1).  A closed surface of n_p flat triangular panels (vertices
 * counter-clockwise seen from the solvent) encloses n_c point charges; the
 * interior has permittivity eps_in, the solvent eps_out.  With one unknown per
 * panel (piecewise constant), collocation at the panel centroids and a
 * quadrature rule on every panel, Eq. ASC becomes the second-kind system
 *
 *     A sigma = b,   A = I + Ehat K',   b = -Ehat (B q),
 *     Ehat = 2 (eps_in - eps_out) / (eps_in + eps_out),
 *     K'_ij = A_j sum_q w_q [-(c_i - y_jq).n_i] / (4 pi |c_i - y_jq|^3),  K'_ii = 0,
 *     (B q)_i = sum_k q_k [-(c_i - x_k).n_i] / (4 pi |c_i - x_k|^3),
 *
 * (the normal derivative of Eq. ASC taken as the interior limit; K'_ii = 0
 * exactly on a flat panel).  sigma is eps_in times the physical induced
 * charge, so the reaction potential of Eq. reac at the charges is
 * phi = C sigma / eps_in, (C s)_k = sum_j s_j A_j sum_q w_q / (4 pi |x_k - y_jq|),
 * and the solvation free energy (Sec. 2.1) is
 *
 *     dG = 1/2 sum_k q_k phi_k = 4 pi * 332.0637 / (2 eps_in) * q.(C sigma)  [kcal/mol].
 *
 * Products with K', B and C run as fast multipole passes (Sec. 2.3: P2M, M2M,
 * M2L, L2L, L2P over an octree plus the near-field P2P panel quadrature).
 *
 * Conventions for every entry point:
 *  - Lengths in Angstrom, charges in e, energies in kcal/mol.
 *  - Array arguments may be host or device pointers (device memory of the
 *    current device, or managed memory); the library detects which.  A device
 *    array is read or written in stream order on the mesh's stream; the call
 *    returns after its results are complete (it synchronises that stream).
 *  - Vectors over panels are in the caller's panel order (length n_p, f64);
 *    vectors over charges are in the caller's charge order (length n_c).
 *  - The caller owns every array it passes; the library copies what it keeps.
 *  - Return value: BEM_OK (0) or a negative BEM_E* code; nothing aborts.
 *    bem_last_error() gives a message for the calling thread's last failure.
 */
#ifndef LIBBEM_BEM_H
#define LIBBEM_BEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define BEM_OK 0
#define BEM_EINVAL (-1)       /* bad argument: NaN/Inf, zero-area panel, eps <= 0, n_p = 0 ... */
#define BEM_ENOMEM (-2)       /* device or host allocation failed */
#define BEM_ECUDA (-3)        /* a CUDA runtime call failed */
#define BEM_ENOCONV (-4)      /* GMRES hit max_iter or stagnated; best iterate written */
#define BEM_ETIMEOUT (-5)     /* a bounded device-side wait ran out */
#define BEM_EUNSUPPORTED (-6) /* option combination not built */

/* ---- options ----------------------------------------------------------- */
#define BEM_MIXED 0 /* FP32 P2P and expansions, FP64 GMRES / epilogues / reductions */
#define BEM_FP64 1  /* every kernel in FP64 (the plain double-precision GPU form) */

#define BEM_BIBEE_CFA 0       /* lambda = -1/2 (Eq. CFA) */
#define BEM_BIBEE_P 1         /* lambda =  0               (Sec. 2.2) */
#define BEM_BIBEE_PLUS_HALF 2 /* lambda = +1/2             (Sec. 2.2) */

#define BEM_FLAG_NO_FAR 1u      /* diagnostics: drop the far field (expansions) */
#define BEM_FLAG_NO_NEAR 2u     /* diagnostics: drop the near field (P2P + table) */
#define BEM_FLAG_NO_NEARTAB 4u  /* diagnostics: skip the near-singular FP64 table */
#define BEM_FLAG_CHECK_CHARGES 8u /* bem_mesh_create rejects (BEM_EINVAL) a charge the surface
                                     does not enclose (winding number from the panels' solid
                                     angles; checked when n_c x n_p x 7 <= 4e10, skipped above) */
#define BEM_FLAG_M2L_REDUCE 16u   /* accepted for compatibility, no effect: the tensor-core M2L
                                     always adds each pair's row into its target cell with
                                     vector reductions (no per-pair buffer) */
#define BEM_FLAG_CHARGE_NEAR_EXACT 32u /* higher-accuracy panel integration of the charges
                                     (Sec. 2.1): in C s, C^T q and grad_x C s every pair of a
                                     charge and a panel whose centroid lies within 2.5 sqrt(A_j)
                                     takes the exact single-layer integral over the flat panel
                                     (FP64) instead of the quadrature rule; the panel vertices
                                     are kept on the device (72 bytes per panel).  Returns
                                     BEM_EUNSUPPORTED if a panel is wider than the charge tree's
                                     neighbour reach. */
#define BEM_FLAG_P2M_FROM_POINTS 64u /* P2M of the quadrature points evaluated from the points
                                     on every product instead of from the per-panel moments
                                     built at mesh creation (the two agree to FP32 rounding;
                                     this form needs no moment storage) */

/* bem_options.near_table */
#define BEM_NEAR_QUADRATURE 1
#define BEM_NEAR_EXACT 2

typedef struct bem_options {
    int precision;     /* BEM_MIXED (default) or BEM_FP64 */
    int p;             /* expansion order, 1..16 (default 10) */
    int leaf_size;     /* target mean panels per non-empty leaf (default 64) */
    int depth;         /* octree leaf level; 0 = choose from leaf_size; -1 = single leaf */
    int quad_points;   /* panel quadrature: 7 (degree-5 rule, default) or 1 (centroid) */
    int gmres_restart; /* GMRES(m) restart length (default 30) */
    int max_iter;      /* total GMRES iterations (default 300) */
    double tol;        /* relative residual |b - A x| / |b| (default 1e-8) */
    unsigned flags;    /* BEM_FLAG_* (default 0) */
    int near_table;    /* near-singular pairs (panel i with the panels whose centroid lies
                          within 2.5 sqrt(A_i)): 1 = corrected to their FP64 quadrature value
                          (default); BEM_NEAR_EXACT = their exact flat-panel integral (solid
                          angle + edge logarithms; higher accuracy, Sec. 2.1); 0 = no
                          correction (diagnostics) */
    int charge_mode;   /* products with B, B^T, C, C^T (charges <-> surface):
                          0 = auto (direct sum when n_c * n_p * quad_points <= 4e10,
                              fast multipole otherwise), 1 = fast multipole, 2 = direct */
    int m2l_mode;      /* translations (M2M, M2L, L2L): 0 = auto (3 when available, else 1),
                          1 = dense real operators grouped by offset class (batched SIMT
                          GEMM), 2 = per-target complex sums (reference form), 3 = as 1
                          with M2L on the tensor cores (tcgen05, 3xTF32; BEM_MIXED, p <= 10) */
    int graph;         /* 1 = replay the K' product as a captured CUDA graph; 0 (default) = launch
                          its kernels on the mesh's two prioritised streams, where the near
                          and far fields overlap better than in a replayed graph */
    int galerkin;      /* 0 (default) = collocation at the centroids; 1 = Galerkin form with
                          piecewise-constant functions (Sec. 2.1): every row of K' and of the
                          right-hand side field averaged over its panel by the quadrature rule,
                          near-singular inner integrals exact.  Product, RHS, solve, energy,
                          BIBEE, the transposed product and the gradients (their transposes
                          place the dipoles at the quadrature points). */
} bem_options;

#define BEM_M2L_AUTO 0
#define BEM_M2L_DENSE 1
#define BEM_M2L_DIRECT 2
#define BEM_M2L_TC 3

#define BEM_CHARGE_AUTO 0
#define BEM_CHARGE_FMM 1
#define BEM_CHARGE_DIRECT 2

typedef struct bem_solve_stats {
    int iterations;      /* GMRES iterations (matrix-vector products inside GMRES) */
    int restarts;
    int converged;       /* 1 if the recurrence residual reached tol */
    double resid;        /* final recurrence residual (relative) */
    double true_resid;   /* |b - A x| / |b| from one extra product */
    double ms_rhs, ms_gmres, ms_total;
} bem_solve_stats;

typedef struct bem_mesh_info {
    int64_t n_p, n_c;
    int depth;             /* leaf level L */
    int p;
    int precision;
    int64_t leaves, cells; /* panel tree */
    int64_t p2p_pairs;     /* exact (target, source point) pairs of one K' near field */
    int64_t m2l_pairs;     /* M2L translations of one K' far field */
    int64_t m2m_pairs;     /* M2M (= L2L) translations of one pass */
    int64_t source_points; /* quadrature points (n_p * quad_points) */
    int64_t near_table_nnz;
    double root_side;      /* root cube side (A) */
    size_t device_bytes;   /* device memory held by the mesh */
    double ms_build;       /* time spent in bem_mesh_create (tree, lists, tables) */
    int64_t p2m_segments;  /* (leaf, panel) segments whose P2M moments were built at mesh
                              creation; 0: P2M works from the quadrature points */
} bem_mesh_info;

typedef struct bem_mesh bem_mesh; /* opaque: owns geometry, trees, lists, scratch */

/* Fill *opt with the defaults above. */
int bem_options_default(bem_options *opt);

/* Build a mesh handle (Sec. 2.1 discretisation, Sec. 2.3 octree).
 *   panels  [n_p][3][3] f64, vertex coordinates, counter-clockwise seen from outside.
 *   charges [n_c][4] f64 rows (x, y, z, q); n_c may be 0 (then no rhs/energy).
 *   eps_in, eps_out > 0.
 *   opt may be NULL (defaults).  stream: a cudaStream_t (NULL = legacy default).
 * Computes panel geometry and quadrature points, Morton keys and sort, the
 * octree, neighbour and interaction lists, translation tables, the FP64
 * near-singular table and the P2M moments of the panels (per leaf and panel,
 * unit density; skipped with BEM_FLAG_P2M_FROM_POINTS or when they would take
 * more than half of the free device memory), all on the device.  Errors: BEM_EINVAL for NaN/Inf
 * coordinates, zero-area panels, eps <= 0, n_p <= 0, bad options.  With the
 * environment variable BEM_TIMING=1 the build steps' wall times are printed
 * to stderr (diagnostics). */
int bem_mesh_create(const double *panels, int64_t n_p, const double *charges, int64_t n_c,
                    double eps_in, double eps_out, const bem_options *opt, void *stream,
                    bem_mesh **out);

/* Release every resource of the handle (NULL is accepted). */
int bem_mesh_destroy(bem_mesh *mesh);

/* Replace the point charges (same or different count); the panel tree is kept,
 * the charge tree and lists and C^T q are rebuilt.  charges [n_c][4] f64. */
int bem_set_charges(bem_mesh *mesh, const double *charges, int64_t n_c);

/* y = A x = x + Ehat K' x  (the BEM operator of Eq. ASC), x, y [n_p] f64.
 * x and y may alias. */
int bem_matvec(bem_mesh *mesh, const double *x, double *y);

/* y = A^T x = x + Ehat K'^T x  (the transposed operator, used by the adjoint). */
int bem_matvec_t(bem_mesh *mesh, const double *x, double *y);

/* b = -Ehat (B q): the right-hand side of Eq. ASC, [n_p] f64. */
int bem_rhs(bem_mesh *mesh, double *b);

/* Solve A sigma = b by restarted GMRES (Sec. 2.1) to opt.tol.
 *   x0: initial guess [n_p] or NULL (zero).  sigma: [n_p] output.
 *   stats may be NULL.  Returns BEM_ENOCONV (sigma still written) when the
 *   iteration budget runs out or the residual stagnates. */
int bem_solve(bem_mesh *mesh, const double *x0, double *sigma, bem_solve_stats *stats);

/* BIBEE (Sec. 2.2, Eq. CFA): K' replaced by lambda I, lambda from `variant`:
 *   sigma_hat = -Ehat / (1 + Ehat lambda) (B q),  then dG as in bem_energy.
 *   sigma_hat [n_p] may be NULL; dG_kcal may be NULL. */
int bem_bibee(bem_mesh *mesh, int variant, double *sigma_hat, double *dG_kcal);

/* Solvation energy of a surface charge (Sec. 2.1, Eq. reac):
 *   phi = C sigma / eps_in at the charges (phi_reac [n_c], may be NULL),
 *   dG = 1/2 q.phi * 4 pi 332.0637  [kcal/mol].
 *   Without phi_reac, dG is formed as (C^T q).sigma with C^T q built once per
 *   charge set (at bem_mesh_create and bem_set_charges) when the charge sums
 *   are direct: the same quantity, one dot product per call. */
int bem_energy(bem_mesh *mesh, const double *sigma, double *dG_kcal, double *phi_reac);

/* Gradient of dG (from the last bem_solve, or a fresh one if none) with
 * respect to the charge values and positions, by the adjoint: solve
 * A^T lam = C^T q, then
 *   d dG/d q_k = kappa/(2 eps_in) [ (C sigma)_k - Ehat (B^T lam)_k ],
 *   d dG/d x_k = kappa/(2 eps_in) q_k [ grad (C sigma)_k - Ehat sum_i lam_i grad_{x_k} B_ik ],
 * kappa = 4 pi 332.0637, each multiplied by grad_out.
 *   dq [n_c] and dx [n_c][3] f64, either may be NULL. */
int bem_energy_backward(bem_mesh *mesh, double grad_out, double *dq, double *dx);

/* Solve many independent meshes (created by bem_mesh_create, possibly of very
 * different sizes) concurrently: right-hand side, GMRES, energy, and the
 * BIBEE/CFA and BIBEE/P bounds (Sec. 2.2) of each.  Host worker threads
 * (`threads`, 0 = 8) each drive one mesh at a time on that mesh's own stream,
 * largest meshes first.  Outputs are indexed like `meshes`:
 *   sigma[i] ([n_p of mesh i] f64, host or device) may be NULL (array or entry),
 *   dG, dG_cfa, dG_p [n] host arrays, each may be NULL; stats [n] may be NULL.
 * Returns the first hard error, else BEM_ENOCONV if any solve did not converge.
 * The molecules run concurrently, each on its own prioritised streams (and,
 * with opt.graph, as its own captured graph) rather than as one persistent
 * launch over all of them (no paper counterpart: the paper solves one system). */
int bem_batch_solve(bem_mesh *const *meshes, int n, int threads, double *const *sigma, double *dG,
                    double *dG_cfa, double *dG_p, bem_solve_stats *stats);

/* Choose opt->leaf_size in {32,64,128,256} and opt->p in {6,8,10} for one
 * geometry: the fastest K' product whose relative error against a p = 12
 * product is at most `target` (inputs as in bem_mesh_create; other fields of
 * *opt are kept).  Builds and times a few trial meshes. */
int bem_autotune(const double *panels, int64_t n_p, const double *charges, int64_t n_c,
                 double eps_in, double eps_out, double target, bem_options *opt);

/* Normal electric field of point charges at given points, for callers that
 * cannot allocate GPU memory (the paper has no counterpart: it is a
 * deployment variant of the direct charge-to-surface product behind
 * bem_rhs).  Callers inside another framework's memory pool, real-time loops
 * that must not touch the allocator, or processes whose device memory is
 * already handed out can call it: it allocates nothing.
 *   field_i = sum_k q_k [-(t_i - x_k).n_i] / (4 pi |t_i - x_k|^3),
 * so -Ehat * field at the panel centroids is the right-hand side of bem_rhs.
 *   targets [n_t][3], normals [n_t][3] (unit), charges [n_c][4] (x, y, z, q),
 *   field [n_t]: all f64 arrays in device memory of the current device (or
 *   managed memory); host pointers and another device's memory: BEM_EINVAL.
 *   stream: cudaStream_t the work is queued on (NULL = legacy default); the
 *   call returns without waiting.
 * Its only scratch is one array inside the library, BEM_NOALLOC_SCRATCH_FLOATS
 * floats (8 MiB) held by every device that loads the library until exit;
 * n_t > BEM_NOALLOC_SCRATCH_FLOATS is rejected with BEM_EINVAL.  All calls on a
 * device share that array and leave their partial sums in it: calls that
 * overlap on the GPU (two streams, two threads) race and must be serialised.
 * The first call on each device looks the array's address (and the device's
 * SM count) up; make that first call before any stream capture. */
#define BEM_NOALLOC_SCRATCH_FLOATS (1 << 21)
int bem_normal_field_noalloc(const double *targets, const double *normals, int64_t n_t,
                             const double *charges, int64_t n_c, double *field, void *stream);

/* Sizes and counts of the handle (tree depth, list sizes, memory). */
int bem_mesh_info_get(const bem_mesh *mesh, bem_mesh_info *info);

/* Clock cycles one device-side pipeline wait of the tensor-core M2L kernel
 * may spin before the call gives up with BEM_ETIMEOUT (default 2e9, about a
 * second; 0 restores the default).  The kernel then leaves cleanly (it waits
 * for its own MMAs, which always finish, and frees its tensor memory), so
 * the mesh stays usable for the next call.  A tiny budget exercises that path
 * from the host.  BEM_EINVAL for a NULL mesh or a negative count. */
int bem_set_wait_budget(bem_mesh *mesh, long long cycles);

/* Cap, in bytes, on the device memory the library's arrays hold in this
 * process (0 = no cap, the default).  An allocation that would pass it fails
 * with BEM_ENOMEM before reaching the CUDA allocator; arrays already held are
 * kept.  Process-wide, for callers that share the GPU with other work. */
int bem_set_device_memory_cap(size_t bytes);

/* Per-phase device time (ms) of the last bem_matvec, measured with CUDA events
 * when enabled by bem_set_profiling(mesh, 1): order P2M, M2M, M2L, L2L, L2P,
 * P2P, epilogue.  times[7]. */
int bem_set_profiling(bem_mesh *mesh, int enable);
int bem_last_phase_ms(const bem_mesh *mesh, double *times);

/* Inside the M2L phase of the last profiled bem_matvec with the tensor-core
 * M2L: device time (ms) of the multipole split (k_split_m), of the
 * tensor-core kernel (k_m2l_tc, which adds the rows into their targets) and
 * a third entry kept at 0 (there is no separate summation kernel).
 * times[3]; zeros if the product had no tensor-core M2L.  BEM_EINVAL if
 * profiling is off. */
int bem_last_m2l_ms(const bem_mesh *mesh, double *times);

/* Inside the P2P phase of the last profiled bem_matvec: device time (ms) of
 * the near field's source strength records (k_strength) and of the
 * near-field kernel itself (k_p2p, with the near-singular table of the
 * collocation product).  times[2]; zeros if the product had no near field.
 * BEM_EINVAL if profiling is off. */
int bem_last_near_ms(const bem_mesh *mesh, double *times);

/* FP32 throughput of the current device in TFLOP/s, measured by chains of
 * packed FP32 fused multiply-adds on every SM (a few milliseconds): the
 * achievable peak of the near-field kernel's arithmetic, for rooflines (the
 * paper has no counterpart).  BEM_EINVAL for a NULL pointer. */
int bem_fp32_peak(double *tflops);

/* Message for the calling thread's last error (static storage, never NULL). */
const char *bem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBBEM_BEM_H */
