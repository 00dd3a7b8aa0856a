/*
 * bchar.h -- C ABI of the GB300 B-char library (libbchar.so).
 *
 * One time step of the ball-approximated characteristics (B-char) method of
 * Cheng & Droniou, "An efficient implementation of mass conserving
 * characteristic-based schemes in 2D and 3D" (arXiv 1908.05834), for the pure
 * advection problem  phi dc/dt + div(u c) = 0  with u.n = 0 on the boundary
 * (Sec 1, eq. advection), on a tensor-product mesh of a box in 2D or 3D:
 *
 *   c^{n+1}_K = sum_M W_KM c^n_M,   W_KM = a_KM / |K|_phi   (Sec 2, eq. phys-inter-ELLAM)
 *
 * where a_KM approximates |M cap F_{-dt}(K)|_phi by balls (Sec 3, eq. ball_int),
 * adjusted by N alternating scalings (Sec 3.2, eq. volAdj) and the
 * mass-conservation minimisation (Sec 3.2, eq. opti_masscons).  Every stage
 * runs in this library's own CUDA kernels on the stream given at creation.
 *
 * Conventions
 *   - Every call returns a bchar_status by value; nothing throws across the ABI.
 *     On error, bchar_last_error(mesh) gives a one-line description.
 *   - Cells are numbered x fastest: k = i + n_x (j + n_y l).
 *   - Face velocities of axis a are numbered the same way with n_a + 1 entries
 *     along axis a (lowest-order Raviart-Thomas degrees of freedom: the
 *     average normal velocity over each face, Sec 1.2 eq. hyp:un).
 *   - Host pointers passed in are read before the call returns and not kept.
 *   - c_in / c_out of bchar_step are DEVICE pointers owned by the caller.
 *   - A mesh handle is used by one host thread at a time.  All device memory
 *     it needs is owned by the handle and released by bchar_destroy.
 */
#ifndef BCHAR_H
#define BCHAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bchar_mesh_s *bchar_mesh_t;

typedef enum {
    BCHAR_OK = 0,
    BCHAR_ERR_INVALID_ARG = 1,   /* bad size, pointer, ordering or option   */
    BCHAR_ERR_OUT_OF_MEMORY = 2, /* a device allocation failed              */
    BCHAR_ERR_CUDA = 3,          /* a CUDA runtime call or kernel failed    */
    BCHAR_ERR_BOUNDARY_FLUX = 4, /* u.n != 0 on the boundary (Sec 1)        */
    BCHAR_ERR_DIVERGENCE = 5,    /* div u != 0 in a cell (Sec 2.2)          */
    BCHAR_ERR_NONFINITE = 6,     /* NaN/Inf in an input                     */
    BCHAR_ERR_NO_VELOCITY = 7,   /* bchar_step before bchar_set_velocity    */
    BCHAR_ERR_CAPACITY = 8       /* a fixed internal limit was exceeded     */
} bchar_status;

/* Arithmetic of the tracking and intersection stages. */
enum { BCHAR_FP64 = 0, BCHAR_FP32_SPLIT = 1 };
/* Storage type of c. */
enum { BCHAR_C_F64 = 0, BCHAR_C_F32 = 1 };

typedef struct {
    int balls_per_axis; /* nb: balls per axis on a cube cell (Sec 4: 4 balls in 2D, 8 in 3D -> 2) */
    int n_scale;        /* N, alternating scalings before the minimisation (Sec 4: N = 10) */
    int precision;      /* BCHAR_FP64: every stage in FP64.  BCHAR_FP32_SPLIT: tracking
                           and ball intersections in FP32, all sums, the scalings, the
                           minimisation and the update in FP64 */
    int substeps;       /* RK4 substeps per step; 0 = smallest s with dt*vmax/s <= cfl*hmin */
    double cfl;         /* 0.5 */
    double drop_tol;    /* entries V_KM < drop_tol |K|_phi are dropped (1e-12) */
    double penalty;     /* eps of the elastic penalty of the minimisation (1e-7), see bchar_step */
    double qp_tol;      /* the minimisation stops when every constraint residual is <= qp_tol of
                           its target (1e-9), the mean complementarity is <= 1e-12 and the
                           stationarity residuals are <= 1e-12 of the largest multiplier */
    int qp_max_iter;    /* cap on conjugate-gradient iterations of one step, all solves (200000) */
    int qp_max_refine;  /* cap on interior-point iterations of one step (300) */
    double div_tol;     /* relative tolerance of the velocity checks (1e-9) */
    int qp_precond;     /* preconditioner of the minimisation's conjugate gradients:
                           1 = aggregation multigrid (default), 0 = Jacobi */
    int qp_warm_start;  /* reserved (0 or 1, default 1; no effect): every minimisation starts
                           from the same centred point, 1 + x = 1, zero constraint multipliers
                           (see bchar_step) */
    int slab_width;     /* entries per row of the assembly's row slab; 0 (default) = 24 in 2D,
                           64 in 3D; wider rows go to the spill area (results are the same) */
} bchar_options;

typedef struct {
    double mass_before;      /* sum_K |K|_phi c^n_K, FP64 (Sec 2.1) */
    double mass_after;       /* sum_K |K|_phi c^{n+1}_K from the FP64 update, before any FP32 rounding */
    double mass_after_stored;/* the same from the stored c_out */
    double max_rel_row_res;  /* max_K |sum_M a_KM - |K|_phi| / |K|_phi  (eq. localmassconsMat) */
    double max_rel_col_res;  /* max_M |sum_K a_KM - |M|_phi| / |M|_phi  (eq. globalmassconsMat) */
    double scale_err;        /* max relative column error after the N scalings */
    double kkt_rel;          /* largest constraint residual / target of the minimisation's result */
    int64_t nnz;             /* non-zeros of A */
    int32_t substeps;        /* RK4 substeps used */
    int32_t cg_iters;        /* conjugate-gradient iterations, all solves of the minimisation */
    int32_t ip_iters;        /* interior-point iterations of the minimisation */
    int32_t qp_converged;    /* 1 if the minimisation met its stopping rule (see qp_tol) */
    int32_t void_balls;      /* tracked balls that met no residing ball */
    int32_t empty_cols;      /* residing cells no tracked ball reached (seeded) */
    int32_t n_at_bounds;     /* entries whose 1 + x ends within 1e-9 of 0 or 2 */
    int32_t kernel_launches; /* kernels launched by this call */
    int32_t amg_levels;      /* levels of the multigrid preconditioner (0 = Jacobi) */
    int32_t amg_coarsest;    /* unknowns on its coarsest level */
    int32_t unbalanced;      /* connected components whose local targets were rescaled (see bchar_step) */
    int32_t row_cap;         /* entries per row of the assembly's row slab: 24 (2D) or 64 (3D); the slab
                              * holds n_c x row_cap x 12 bytes */
    int32_t spill_rows;      /* rows wider than the slab, assembled a second time into a spill area of
                              * their exact total length */
    int32_t max_row_len;     /* entries of the widest row of A */
    /* Milliseconds on the handle's stream (CUDA events) per stage of this call:
     * [0] tracking, [1] intersections and row assembly (with empty-column
     * seeding), [2] compaction, column view and target balancing, [3] the N
     * scalings, [4] the minimisation (multigrid set-up and CG), [5] bounds,
     * column fix and W, [6] update and masses, [7] the whole call from the
     * first to the last stage.  Host round trips inside a stage count in it. */
    float ms_stage[8];
} bchar_step_info;

/* Fill *opt with the defaults listed above. */
void bchar_default_options(bchar_options *opt);

/* Create a mesh: the tensor-product partition of the box
 * [coords[0][0], coords[0][n0]] x ... (Sec 1.2), porosity phi (Sec 1.2,
 * eq. assump.global: piecewise constant, > 0) and its balls (Sec 3: n_K equal
 * balls of radius min width / (2 nb), tightly packed, nb per axis on a cube).
 *   dim       2 or 3
 *   n_cells   dim counts, each >= 1 (and n_c = prod <= 2^31 - 1)
 *   coords    dim HOST arrays of n_cells[a] + 1 strictly increasing doubles
 *   phi       HOST array of n_c doubles, finite and > 0, x fastest
 *   opt       NULL for the defaults
 *   stream    cudaStream_t all work of this handle is ordered on (NULL = legacy default)
 *   out       receives the handle (NULL on failure)
 * Errors: INVALID_ARG, NONFINITE, OUT_OF_MEMORY, CUDA. */
bchar_status bchar_create_mesh(int dim, const int64_t *n_cells, const double *const *coords,
                               const double *phi, const bchar_options *opt, void *stream,
                               bchar_mesh_t *out);

/* Set the velocity u^{(n+1)} of the next step (Sec 1.2, eq. hyp:un): dim
 * arrays of face-normal velocities (layout above, (n_a + 1) prod_{b != a} n_b
 * doubles each), HOST pointers when on_device = 0, DEVICE pointers when 1
 * (read on the handle's stream).  Checks that u.n = 0 on the boundary
 * (Sec 1) and that every cell's net flux vanishes (div u = 0, Sec 2.2), both
 * relative to the largest face velocity times div_tol.
 * Errors: INVALID_ARG, NONFINITE, BOUNDARY_FLUX, DIVERGENCE, CUDA (the
 * previous velocity is then discarded). */
bchar_status bchar_set_velocity(bchar_mesh_t m, const double *const *face_u, int on_device);

/* One B-char time step of length dt > 0 (Algorithm 1 and eq. phys-inter-ELLAM):
 *   1. every ball centre (and, if phi is not constant, the 2 dim points on
 *      its axes at distance r) is tracked back along dF/dt = u/phi over dt by
 *      classical RK4 (Sec 2 eq. charac, Sec 3 eq. rTrackedBall);
 *   2. a^(0)_KM = V_{K,M} from the closed-form ball intersections
 *      (Sec 3.1, eq. fracMaterial, eq. ball_int);
 *   3. consistent targets: on a connected component of A's pattern (row i
 *      and column j linked by every non-zero a_ij) whose local targets
 *      sum_rows |K_i|_phi differ from its global ones sum_cols |M_j|_phi (the
 *      balls can cause this), the local targets are scaled by their ratio;
 *      then N alternating column/row scalings (Sec 3.2, eq. volAdj);
 *   4. the minimisation of Sec 3.2 (eq. opti_masscons) with the paper's bounds
 *      0 <= 1 + x <= 2 inside it, read as: minimise 1/2 x.x + sum_l h(v_l) over
 *      the bounds, v_l the relative violation of each of the 2 n_c mass
 *      constraints and h quadratic (v^2 / (2 eps^2), eps = penalty) up to
 *      |v| = 1e-6 and linear beyond.  Where the paper's problem has a solution
 *      this is that solution up to residuals eps^2 y_l; where the balls make
 *      the constraints contradictory (a cell whose only tracked overlap is a
 *      smaller neighbour), the total relative violation is the least the
 *      bounds allow.  Solved by a primal-dual interior-point method whose
 *      linear systems are solved by multigrid-preconditioned conjugate
 *      gradients; then every column scaled to |M|_phi so that global mass is
 *      conserved to rounding.  If the minimisation reaches qp_max_refine or
 *      qp_max_iter before its stopping rule, the step still completes from
 *      the last iterate (the bounds and global mass hold at any iterate), the
 *      status is OK and info->qp_converged = 0;
 *   5. c_out = W c_in (eq. phys-inter-ELLAM), FP64 accumulation.
 * c_in, c_out: DEVICE arrays of n_c values of type c_dtype, caller-owned, not
 * aliased.  info: optional (NULL), written on return.  The call returns when
 * the step has finished on the device.
 * Errors: INVALID_ARG, NO_VELOCITY, OUT_OF_MEMORY, CAPACITY, CUDA. */
bchar_status bchar_step(bchar_mesh_t m, double dt, const void *c_in, void *c_out, int c_dtype,
                        bchar_step_info *info);

/* Release the handle and all its device memory (NULL is ignored). */
void bchar_destroy(bchar_mesh_t m);

/* Static text of a status code. */
const char *bchar_status_string(bchar_status s);

/* Detail of the last error on this handle ("" if none). */
const char *bchar_last_error(bchar_mesh_t m);

/* Number of cells n_c and of balls of the mesh. */
int64_t bchar_cell_count(bchar_mesh_t m);
int64_t bchar_ball_count(bchar_mesh_t m);

/* Copy one matrix of the last step to HOST buffers in CSR form (rows =
 * tracked cells K, columns = residing cells M, columns sorted in each row):
 * which = 0: A^(0) (after seeding empty columns), 1: A^(N) after the
 * scalings, 2: the final a_KM.  row_ptr gets n_c + 1 entries; cols / vals get
 * nnz entries (cap = their capacity; *nnz_out receives nnz).  Errors:
 * INVALID_ARG (no step yet, bad which), CAPACITY (cap < nnz), CUDA. */
bchar_status bchar_export_matrix(bchar_mesh_t m, int which, int64_t *row_ptr, int32_t *cols,
                                 double *vals, int64_t cap, int64_t *nnz_out);

/* Copy the tracked balls of the last step to HOST buffers: pos[3 b + a] the
 * tracked centre (absolute coordinates; a = 2 is 0 in 2D), rhat[b] the
 * tracked radius, balls b of cell K numbered consecutively from
 * ball_offset[K] (ball_offset: n_c + 1 entries).  cap = capacity in balls.
 * Errors: INVALID_ARG, CAPACITY, CUDA. */
bchar_status bchar_export_tracked(bchar_mesh_t m, double *pos, double *rhat, int64_t *ball_offset,
                                  int64_t cap);

/* Stages that bchar_time_stage can replay. */
enum {
    BCHAR_STAGE_CG_MATVEC = 0, /* one product with A-hat A-hat^T + W (the minimisation's inner loop) */
    BCHAR_STAGE_UPDATE = 1,    /* c^{n+1} = W c^n and the mass sums */
    BCHAR_STAGE_ASSEMBLE = 2,  /* ball intersections and row assembly into the slab */
    BCHAR_STAGE_TRACK = 3,     /* RK4 tracking of all balls */
    BCHAR_STAGE_SMOOTH = 4,    /* one damped-Jacobi sweep of the multigrid's finest level */
    BCHAR_STAGE_SCALING = 5,   /* one column and one row scaling of eq. volAdj (on scratch copies) */
    BCHAR_STAGE_VCYCLE = 6     /* one V-cycle of the multigrid preconditioner (the last one built) */
};

/* Measurement aid: replay the kernel of one stage `reps` times on the data of
 * the last step, on the handle's stream, and return the mean duration of one
 * launch in milliseconds (CUDA events around the replays).  CG_MATVEC, UPDATE,
 * SMOOTH and VCYCLE are replayed from one CUDA graph of `reps` launches
 * (captured on a private stream), so that host launch overhead is not
 * measured; SCALING too (it writes the scaling factors, which the step no
 * longer needs).  VCYCLE (a chain of kernels, one per pass and level) needs a
 * step that built the multigrid hierarchy, like SMOOTH.  The replays do
 * not change the result of the last step (exports stay valid) except that
 * BCHAR_STAGE_TRACK overwrites the tracked balls with the same values.
 * Errors: INVALID_ARG (no step yet, bad stage, reps < 1), CUDA. */
bchar_status bchar_time_stage(bchar_mesh_t m, int stage, int reps, float *mean_ms);

/* The porous mass sum_K |K|_phi c_K (the quantity bchar_step_info reports as
 * mass_before / mass_after), for callers that must not allocate device memory:
 * a time-stepping loop with a fixed device-memory budget, a framework that
 * hands out memory only from its own pool, or code that must not take the
 * implicit synchronisation of cudaMalloc/cudaFree in the middle of a step.
 * The paper has no counterpart; this is a service of the library.
 *   volphi   DEVICE array of n values |K|_phi (FP64), caller-owned
 *   c        DEVICE array of n values (c_dtype BCHAR_C_F64 or BCHAR_C_F32), caller-owned
 *   n        1 <= n <= 16 777 216 (2^24); larger n returns BCHAR_ERR_CAPACITY
 *   mass_out DEVICE pointer to one double, written by the call
 *   stream   cudaStream_t the work is ordered on (NULL = legacy default)
 * Allocates nothing: the per-block partial sums use a fixed 8 KB array inside
 * the library's device memory, held by every GPU that loads the library until
 * the process exits.  The first call on a device looks up that array's
 * address (with the device current), so make the first call before any
 * stream capture.  All calls share the array: calls that overlap on the GPU
 * (different streams, no ordering between them) race and may return wrong
 * sums; order them on one stream.  Returns when the work is queued.
 * Errors: INVALID_ARG, CAPACITY, CUDA. */
bchar_status bchar_mass_noalloc(const double *volphi, const void *c, int c_dtype, int64_t n, double *mass_out,
                                void *stream);

/* Like bchar_set_velocity, with every face velocity multiplied by `scale`
 * (finite; 0 is allowed and stops the flow) on the device after the copy:
 * for fields of the form u(x) g(t), the caller passes u once per step with
 * the factor g(t^n + dt/2) and needs no scaled copy of its own.  The checks
 * (boundary flux, divergence) apply to the scaled field.
 * Errors: as bchar_set_velocity; INVALID_ARG for a non-finite scale. */
bchar_status bchar_set_velocity_scaled(bchar_mesh_t m, const double *const face_u[3], int on_device, double scale);

/* Device memory held by the handle now and at most so far (bytes; every
 * buffer the library allocated for it).  Either pointer may be NULL, not both.
 * Errors: INVALID_ARG. */
bchar_status bchar_device_bytes(bchar_mesh_t m, int64_t *now, int64_t *peak);

/* A-priori estimate (bytes) of the device memory a handle created with these
 * arguments will hold after its steps, for admission control before any
 * allocation: per cell (mesh arrays, minimisation vectors, row slab,
 * multigrid), per ball (the tight packing, counted here from the widths)
 * and per matrix entry, with the entries bounded by a 3^d neighbourhood per
 * row (9 in 2D, 27 in 3D), plus 10 %.  Rows wider than the slab's 24 (2D)
 * or 64 (3D) entries are held at their exact length in a spill area, which the
 * per-entry count covers.  Host only; no GPU work.  coords as for
 * bchar_create_mesh; opt NULL = defaults.
 * Errors: INVALID_ARG. */
bchar_status bchar_estimate_device_bytes(int dim, const int64_t n_cells[3], const double *const coords[3],
                                         const bchar_options *opt, int64_t *bytes);

/* One time step of `count` independent handles at once (the paper has no
 * counterpart; it steps one mesh).  Instance i is bchar_step(meshes[i],
 * dt[i], c_in[i], c_out[i], c_dtype[i], infos ? &infos[i] : NULL), with the
 * same arguments, rules and result, bitwise; the instances run concurrently
 * from up to max_workers host threads of the library (<= 0: 16), largest
 * mesh first, each on its handle's own stream.  Give every handle its own
 * stream: handles that share one still give correct results but run one after
 * the other on the GPU.  The handles must be distinct (a handle is used by
 * one thread at a time) and none may be in use elsewhere during the call.
 * Returns when every instance has finished; the current device of the calling
 * thread is kept.
 *   statuses  HOST array of count statuses (nullable), one per instance
 *   infos     HOST array of count bchar_step_info (nullable)
 * Returns OK, or the first failing instance's status (in index order); the
 * other instances still ran.  Errors: INVALID_ARG (count < 0, a NULL array or
 * handle, a handle listed twice), CUDA, OUT_OF_MEMORY (host threads). */
bchar_status bchar_step_batch(int count, const bchar_mesh_t *meshes, const double *dt, const void *const *c_in,
                              void *const *c_out, const int *c_dtype, bchar_step_info *infos,
                              bchar_status *statuses, int max_workers);

#ifdef __cplusplus
}
#endif

#endif /* BCHAR_H */
