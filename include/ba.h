/* ba.h -- C ABI of the B300 holistic bundle-adjustment library (libba.so).
 *
 * One Levenberg-Marquardt (LM) step of the unified bundle adjustment of
 * "Stable and Scalable Bundle Adjustment of Holistic 3D Structures":
 * cameras and groups (planes, vanishing points) form the kept set A = C u G
 * (Section 3.2, Eq. 5); points and lines are features, eliminated by the Schur
 * complement S = H_aa - H_af H_ff^-1 H_fa (Eq. 3 / Eq. 5), which is solved by
 * block-Jacobi preconditioned CG; the features are then back-substituted.
 *
 * Residual kinds (one observation record per residual):
 *   BA_OBS_POINT        point reprojection, Eq. 1 / Eq. 4          meas: 2 (distorted pixels)
 *   BA_OBS_LINE         line reprojection rho in R^4, Eq. 4      meas: 4 (segment endpoints, undistorted)
 *   BA_OBS_PLANE_POINT  plane-induced point residual, Eq. 7      meas: none (other = plane id)
 *   BA_OBS_PLANE_LINE   plane-induced line residual, Eq. 8       meas: 4 (segment; other = plane id)
 *   BA_OBS_VP           VP angular residual d x v, Eq. 6         meas: none (cam = -1, other = VP id)
 *   BA_OBS_P2L          wireframe point -> observed line, Eq. 11 meas: 4 (partner segment; other = line id)
 *   BA_OBS_L2P          wireframe line -> observed point, Eq. 12 meas: 2 (partner point, undistorted)
 * Plane projections of points and Pluecker lines follow Appendix B.  Weights and
 * Cauchy scales default to the cost-balancing values of Appendix C; the cost is
 * E = 1/2 sum w a^2 ln(1 + |r|^2/a^2), and termination uses the relative change
 * of the pixel-space part only (Section 3.5).
 *
 * Conventions.
 *   Memory: every pointer argument is host memory when mem == BA_MEM_HOST and
 *     device memory of the current CUDA device when mem == BA_MEM_DEVICE.  Input
 *     arrays are copied; the caller keeps ownership of its buffers.  The library
 *     owns all device memory it allocates (through the optional allocator hooks
 *     of ba_options, else cudaMalloc) and frees it in ba_destroy.
 *   Indices: 0-based int32, per type (point ids, line ids, plane ids, VP ids).
 *     They, and the finiteness of the measurements, are validated when the
 *     structure is frozen (first step); an out of range index or a non-finite
 *     measurement returns BA_ERR_ARG there.
 *   Freezing: adding data after the first ba_lm_step / ba_solve / ba_build_reduced
 *     returns BA_ERR_STATE.
 *   Errors: no exception or abort crosses the ABI.  Every call returns a
 *     ba_status; ba_last_error() gives a message for the last failure of that
 *     problem.  After BA_ERR_CUDA the problem can still be destroyed.
 *   Streams: all device work runs on options.cuda_stream (NULL = legacy default
 *     stream); calls return after the work they report on has finished.
 *   Layout of parameters: camera quat_t n x 7 = (qw, qx, qy, qz, tx, ty, tz),
 *     world -> camera (x_c = R(q) X + t, +z forward); intrinsics n x 3 = (f, k1, k2);
 *     principal points n x 2.  Points n x 3.  Lines n x 6 Pluecker (d, m), m . d = 0
 *     (rescaled internally so that |d| = 1).  Planes n x 4 (n, w), plane n.x + w = 0.
 *     VPs n x 3 directions.
 *   Limits: a feature may be associated with at most one plane and one VP.
 */
#ifndef BA_H
#define BA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_problem ba_problem;

typedef enum {
  BA_OK = 0,
  BA_ERR_ARG = -1,      /* invalid argument (null pointer, bad kind, index out of range, size limit) */
  BA_ERR_STATE = -2,    /* call not allowed in the current state (e.g. adding after freezing) */
  BA_ERR_CUDA = -3,     /* a CUDA runtime call failed */
  BA_ERR_OOM = -4,      /* device or host allocation failed */
  BA_ERR_NUMERIC = -5,  /* non-finite cost or a linear-algebra breakdown that damping could not fix */
  BA_ERR_TIMEOUT = -6   /* a bounded device-side wait ran out */
} ba_status;

typedef enum { BA_MEM_HOST = 0, BA_MEM_DEVICE = 1 } ba_mem;
typedef enum { BA_FP64 = 0, BA_MIXED = 1 } ba_precision;
typedef enum { BA_PRECOND_BLOCK_JACOBI = 0, BA_PRECOND_LEARNED = 1 } ba_precond;
typedef enum { BA_POINT = 0, BA_LINE = 1 } ba_feature_kind;
typedef enum {
  BA_PLANE = 0, BA_VP = 1,
  BA_SPHERE = 2,     /* n x 4: centre c, radius r > 0 (Appendix B; radius updated in log space) */
  BA_CYLINDER = 3,   /* n x 7: axis as a Pluecker line (d, m), m . d = 0 (rescaled to |d| = 1), radius r > 0 */
  BA_CONE = 4,       /* n x 7: apex a, axis direction d (normalised), half-angle in (0, pi/2) */
  BA_ELLIPSOID = 5,  /* n x 10: unit quaternion (w, x, y, z) of R (local -> world), centre c, semi-axes s > 0 */
  BA_CUBOID = 6      /* n x 10: unit quaternion of R, face offsets d_0..d_5 (faces n_i . x = d_i and -n_i . x =
                        d_{i+3} with n_i = R e_i); both 9-parameter groups are two entities of A each */
} ba_group_kind;
typedef enum { BA_REL_ORTHOGONAL = 0, BA_REL_PARALLEL = 1 } ba_relation_type;
typedef enum {
  BA_OBS_POINT = 0, BA_OBS_LINE = 1, BA_OBS_PLANE_POINT = 2, BA_OBS_PLANE_LINE = 3,
  BA_OBS_VP = 4, BA_OBS_P2L = 5, BA_OBS_L2P = 6,
  BA_OBS_PLANE_POINT3D = 7,   /* direct 3D point-to-plane distance n.X + w (no camera, no measurement) */
  BA_OBS_PLANE_LINE3D = 8,    /* direct 3D line-to-plane distances n.d and n.(d x m) + w (|d| = 1; no camera) */
  /* group-induced point residuals of the other group types (Eq. 7 with the projections of Appendix B): a point
   * observed in a camera, other = the sphere / cylinder / cone id; no measurement */
  BA_OBS_SPHERE_POINT = 9, BA_OBS_CYLINDER_POINT = 10, BA_OBS_CONE_POINT = 11,
  BA_OBS_ELLIPSOID_POINT = 12, BA_OBS_CUBOID_POINT = 13,
  /* 3D wireframe endpoint distance X x d - m of a point X to a line (d, m), |d| = 1 (the form Section 3.3 sets
   * against Eq. 11 / Eq. 12): feature = the line id, other = the point id; no camera, no measurement.  Every
   * point it names becomes a 3-value entity of the reduced system (its residuals are not eliminated with
   * it); not together with cam_dof = 9 or the sphere ... cuboid groups, nor in ba_solve_batch (BA_ERR_ARG) */
  BA_OBS_WIREFRAME3D = 14,
  /* Eq. 8 for a line on a cuboid: the line projected onto the cuboid's face nearest the line's point closest to
   * the cuboid's centre (Appendix B); other = the cuboid id, meas: 4 (the segment, as BA_OBS_PLANE_LINE) */
  BA_OBS_CUBOID_LINE = 15
} ba_obs_kind;

typedef struct ba_options {
  int precision;            /* ba_precision: BA_FP64 everything in double; BA_MIXED: Jacobians, Schur and
                               SpMV in float, landmark inverses, damping, cost and the accept test in double */
  double w_point, w_line;   /* loss weights of R1 / R2 (1.0) */
  double w_group;           /* plane-induced residuals R3 / R4 (0.5) */
  double w_wire;            /* wireframe residuals R6 / R7 (0.1) */
  double w_vp;              /* VP angular residual R5 (5e3) */
  double cauchy_px;         /* Cauchy scale of pixel residuals (1.0) */
  double cauchy_vp;         /* Cauchy scale of the VP residual (0.2) */
  double lambda0;           /* initial LM damping (1e-4) */
  double lambda_min, lambda_max; /* damping clamp (1e-12, 1e12) */
  double min_gain;          /* accept when gain ratio > min_gain (1e-3) */
  double rel_cost_tol;      /* stop on an accepted step with |dE_px|/E_px < tol (1e-6) */
  int max_lm_iters;         /* ba_solve iteration cap (20) */
  double pcg_rel_tol;       /* PCG stop: |r_k| <= tol |b| (1e-6) */
  int pcg_max_iters;        /* PCG cap (1000) */
  int precond;              /* ba_precond */
  void* cuda_stream;        /* cudaStream_t to run on (NULL = default stream) */
  void* (*dev_alloc)(size_t bytes, void* ctx);   /* optional device allocator (e.g. the framework's caching allocator);
                                                    must return 256-byte aligned blocks, as cudaMalloc does: a
                                                    misaligned block is freed again and the call fails (BA_ERR_OOM) */
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  long long wait_budget_cycles; /* bound, in clock64 cycles, on each wait at a grid barrier of the persistent
                                   PCG (2e9, about a second): a wait that runs out ends the solve, and the step
                                   returns BA_ERR_TIMEOUT with the problem still usable.  The waits for the bulk
                                   copies of S into shared memory have a fixed bound instead: a copy always
                                   completes, and a kernel never leaves while one is in flight */
  double mixed_lambda_floor; /* BA_MIXED only: an extra lower bound of the damping (0 = none, the default).  An
                                earlier float Schur form needed 1e-6; with the whitened form the floor only slowed
                                the slow tail of the iteration (measured at 2000 cameras) */
  double w_rel;             /* loss weight of the inter-group relations (5e3, the VP term's) */
  double cauchy_rel;        /* Cauchy scale of the inter-group relations (0.2, the VP term's) */
  int batch_ctas_per_window; /* ba_solve_batch, read from windows[0]: 0 = chosen by the autotuner (or 1); 1, 2 or 4
                                = every window on a thread-block cluster of that many CTAs (256 threads each).  The
                                autotuner may also run only the largest windows on clusters and the rest on single
                                CTAs of the same launch */
  double w_group3d;         /* loss weight of the direct 3D plane distances (1.0; the form Section 3.2 sets against
                               the group-induced residuals, weighed 1 to 1000 in Table 5).  Not in E_px */
  double cauchy_3d;         /* their Cauchy scale, in scene units (1.0) */
  int cam_dof;              /* 6 (default): camera blocks refine the pose, f, k1, k2 are held constant; 9: f, k1, k2
                               are refined too (Section 3.1, K_c(i)), as intrinsics entities of the reduced system
                               (3 values each, one per camera unless ba_set_intrinsics shares them); their
                               increments are additive, and the principal point stays constant.  Problems with
                               refined intrinsics keep the full 6 x 6 storage of S and are not supported by
                               ba_solve_batch (BA_ERR_ARG there) */
  double w_wire3d;          /* loss weight of the 3D wireframe endpoint distance (1.0; Cauchy scale cauchy_3d).
                               Not in E_px */
} ba_options;

/* Per-LM-step report. */
typedef struct ba_step_report {
  double cost, cost_px;         /* E and E_px at the current parameters (before the step) */
  double cost_new, cost_px_new; /* at the candidate x (+) delta */
  double pred;                  /* predicted decrease -g.delta - 1/2 delta^T H delta */
  double gain;                  /* (cost - cost_new) / pred */
  double lambda;                /* damping used for this step */
  double pcg_rel;               /* final relative PCG residual |r_k| / |b| */
  int pcg_iters;
  int accepted;
  int converged;                /* accepted with |dE_px|/E_px < rel_cost_tol, or rejected at lambda_max (no step
                                   lowers the cost at the working precision) */
  int relinearized;             /* 1 if the Jacobians were recomputed for this step */
  float ms_linearize, ms_schur, ms_pcg, ms_update;  /* device time per phase */
  /* device time per kernel stage, measured with CUDA events on the problem's stream:
   * [0] derive + linearize (K1; 0 when the step reuses the Jacobians), [1] landmark inverse and whitening
   * (K2), [2] Schur work units and packed small blocks (K3a), [3] Schur diagonal / split-block sums (K3b),
   * [4] block-Jacobi (K4), [5] PCG (K5/K6, one cooperative launch), [6] back-substitution (K7),
   * [7] candidate (K8a), [8] cost (K8b), [9] decision (K9) */
  float ms_kernel[10];
  int n_launches;               /* CUDA kernels this step launched */
  int precond_fallbacks;        /* learned preconditioner: blocks that fell back to block-Jacobi (-1: not used) */
} ba_step_report;

typedef struct ba_solve_report {
  int iters, converged, accepted_steps, total_pcg_iters;
  double cost0, cost, cost_px;
  double ms_structure;          /* one-time structure build (analogue of symbolic analysis) */
  double ms_total;              /* wall time of the whole solve */
  double ms_window;             /* ba_solve_batch: this window's own device time on its CTA (global timer) */
} ba_solve_report;

/* Fill *o with the defaults listed above. */
void ba_default_options(ba_options* o);

/* Create an empty problem.  opts may be NULL (defaults).  *out receives the handle. */
ba_status ba_create(const ba_options* opts, ba_problem** out);
/* Free every resource of the problem (NULL is allowed). */
void ba_destroy(ba_problem* p);
const char* ba_last_error(const ba_problem* p);

/* Cameras (Section 3.1: C_i = (K, R_i, t_i)): quat_t n x 7, f_k1_k2 n x 3, pp n x 2 (principal point, always held
 * constant; f, k1, k2 are held constant too unless cam_dof = 9), fixed: optional n bytes, a bit mask of pose increment components held
 * constant (bits 0-2 rotation dw, 3-5 translation dt; 0x3F holds the whole pose), used to fix the gauge.
 * Appends; ids continue. */
ba_status ba_add_cameras(ba_problem* p, int64_t n, int mem, const double* quat_t, const double* f_k1_k2,
                         const double* pp, const uint8_t* fixed);
/* Features (Section 3.2): kind BA_POINT (n x 3) or BA_LINE (n x 6 Pluecker). */
ba_status ba_add_features(ba_problem* p, int kind, int64_t n, int mem, const double* params);
/* Groups (Section 3.2-3.3, Appendix B, Table 6): kind BA_PLANE (n x 4), BA_VP (n x 3), BA_SPHERE (n x 4),
 * BA_CYLINDER (n x 7), BA_CONE (n x 7), BA_ELLIPSOID (n x 10) or BA_CUBOID (n x 10), layouts at ba_group_kind.
 * A feature may belong to at most one positional group (a plane, sphere, cylinder, cone, ellipsoid or cuboid).
 * The groups other than planes and VPs keep the full 6 x 6 storage of S and are not supported by
 * ba_solve_batch or together with cam_dof = 9 (BA_ERR_ARG).  ba_get_groups returns the add layouts (a
 * 9-parameter group's quaternion with w >= 0). */
ba_status ba_add_groups(ba_problem* p, int kind, int64_t n, int mem, const double* params);
/* Inter-group relations (Section 3.2, Inter-Group Relations; Appendix C, Manhattan / Atlanta world): n
 * relations between two group directions, each a plane normal (kind BA_PLANE) or a VP direction (BA_VP).
 * kind_a, a, kind_b, b, type: n int32 each (type BA_REL_ORTHOGONAL: residual a.b, the cosine of the angle;
 * BA_REL_PARALLEL: residual a x b, its sine as a vector).  Both are angular: weight w_rel and Cauchy scale
 * cauchy_rel, in E but not in the pixel cost E_px.  They involve only group parameters, so they add to the
 * group-group blocks of S (H_gg) and to g_g alone.  Indices are validated when the structure is frozen
 * (BA_ERR_ARG for an unknown kind or type, an id out of range, or a relation of a group with itself).
 * Appends; not supported by ba_solve_batch (BA_ERR_ARG there). */
ba_status ba_add_relations(ba_problem* p, int64_t n, int mem, const int32_t* kind_a, const int32_t* a,
                           const int32_t* kind_b, const int32_t* b, const int32_t* type);
/* Refined intrinsics shared by camera model (Section 3.1: image i uses the intrinsics K_c(i) of its camera model
 * c(i)); only with cam_dof = 9 (BA_ERR_ARG otherwise).  n_intr entities with initial values f_k1_k2 (n_intr x 3)
 * and, for every camera of the problem (n_cams, which must equal the number of cameras added when the structure
 * is frozen, else BA_ERR_ARG there), its entity in [0, n_intr) (intr_of_cam, n_cams int32; validated here).  A
 * camera's own f, k1, k2 from ba_add_cameras are then replaced by its entity's values.  Without this call,
 * cam_dof = 9 gives every camera its own entity, starting from its ba_add_cameras values.  A later call
 * replaces an earlier one; not allowed after freezing (BA_ERR_STATE). */
ba_status ba_set_intrinsics(ba_problem* p, int64_t n_intr, int mem, const double* f_k1_k2,
                            const int32_t* intr_of_cam, int64_t n_cams);
/* Residual records of one kind: cam (n; ignored for BA_OBS_VP and the 3D plane kinds, may be NULL), feature (n), other (n; group id or
 * partner feature id, may be NULL for kinds without one), meas (n x meas_dim(kind), may be NULL when 0). */
ba_status ba_add_observations(ba_problem* p, int kind, int64_t n, int mem, const int32_t* cam,
                              const int32_t* feature, const int32_t* other, const double* meas);

/* One LM iteration (linearise, damp, eliminate, PCG, back-substitute, evaluate, accept/reject). */
ba_status ba_lm_step(ba_problem* p, ba_step_report* out);
/* LM until converged or max_lm_iters.  out may be NULL. */
ba_status ba_solve(ba_problem* p, ba_solve_report* out);

/* Current parameters, same layouts as the add calls; out arrays sized for all entities of that kind. */
ba_status ba_get_cameras(ba_problem* p, int mem, double* quat_t);
ba_status ba_get_features(ba_problem* p, int kind, int mem, double* params);
ba_status ba_get_groups(ba_problem* p, int kind, int mem, double* params);
/* Current f, k1, k2 of every camera (n_cams x 3; with refined intrinsics, its entity's values). */
ba_status ba_get_intrinsics(ba_problem* p, int mem, double* f_k1_k2);
/* LM state (lambda, nu) for checkpoint / resume. */
ba_status ba_get_lm_state(ba_problem* p, double* lambda_nu);
ba_status ba_set_lm_state(ba_problem* p, const double* lambda_nu);

/* Cost (E, E_px) at the current parameters (FP64). */
ba_status ba_eval_cost(ba_problem* p, double* cost, double* cost_px);

/* ln(1 + x) as the FP64 cost pass evaluates it in the Cauchy loss a^2 ln(1 + |r|^2 / a^2) (Section 3.5,
 * Appendix C): a table-driven logarithm (Tang, ACM TOMS 1990) whose table the library fills once per device.
 * x (n values) and y (n values, output) are DEVICE arrays of the current device; runs on cuda_stream (NULL =
 * default stream) and returns after the work has finished.  x >= 0 is the range the cost uses; other values
 * go to the CUDA math library's log1p.  BA_ERR_ARG for n < 0 or a null array, BA_ERR_CUDA if a CUDA call fails.
 * An inspection call for tests of the cost's accuracy. */
ba_status ba_eval_log1p(int64_t n, const double* x, double* y, void* cuda_stream);

/* Measured FMA throughput of the current device, the denominator of the ALU rooflines: precision BA_MIXED
 * measures the FP32 pipe, BA_FP64 the FP64 pipe.  *tflops receives 2 x FMAs per second / 1e12 (the best of
 * three timed launches after a warm-up launch, each thread running eight independent FMA chains).  Runs on
 * cuda_stream (NULL = default stream); allocates and frees a small device buffer.  BA_ERR_ARG for a bad
 * precision or a null pointer, BA_ERR_CUDA if a CUDA call fails.  Not part of the paper's method: a probe for
 * reporting achieved fractions of the arithmetic pipes. */
ba_status ba_measure_fma_rate(int precision, double* tflops, void* cuda_stream);

/* Build the damped reduced system S, b at damping lambda (linearising if needed) without stepping. */
ba_status ba_build_reduced(ba_problem* p, double lambda);
/* Sizes of the reduced system: number of A entities (block rows, each 6 wide, in the order cameras, planes,
 * VPs, intrinsics entities; plane and intrinsics blocks use 3, VP blocks 2 of the 6, the rest are padding with
 * a unit diagonal) and number of stored 6x6 blocks (both triangles). */
ba_status ba_reduced_size(ba_problem* p, int64_t* n_block_rows, int64_t* nnz_blocks);
/* Copy the last reduced system to host: row_ptr (n_block_rows+1), cols (nnz_blocks), vals (nnz_blocks x 36,
 * row-major 6x6, double) and b (n_block_rows x 6).  Any pointer may be NULL. */
ba_status ba_export_reduced_system(ba_problem* p, int32_t* row_ptr, int32_t* cols, double* vals, double* b);
/* Solve the last reduced system by PCG and back-substitute: per-entity increments to host arrays
 * (cams n x 6 as (dw, dt), planes n x 3, vps n x 2, points n x 3, lines n x 4); NULL skips an output. */
ba_status ba_compute_step(ba_problem* p, double* dcam, double* dplane, double* dvp, double* dpoint,
                          double* dline, int* pcg_iters, double* pcg_rel, double* pred);
/* The intrinsics part of the step that ba_compute_step or ba_lm_step computed last: per intrinsics entity its
 * (df, dk1, dk2) (n_intr x 3; nothing to copy without refined intrinsics). */
ba_status ba_get_step_intrinsics(ba_problem* p, double* dk);
/* Number of intrinsics entities in the reduced system (0 with cam_dof = 6).  Freezes the structure. */
ba_status ba_intrinsics_count(ba_problem* p, int64_t* n_intr);

/* Batched local windows: solve n independent problems (windows) with lm_iters LM iterations each, all in one
 * persistent kernel launch captured in a CUDA graph (local bundle adjustment after every registered image
 * dominates incremental SfM, Section 4 / Appendix A.2).  Every window is a problem built with the calls above;
 * all windows must use the same precision and device, and run on the stream of windows[0].  A CTA (or a
 * thread-block cluster of CTAs, which splits the window's features, Schur units and reduced-system rows over
 * its CTAs) takes the next window from a device queue (largest first) and runs its iterations on the device (the same linearise /
 * invert / Schur / PCG / back-substitute / cost / decide steps as ba_lm_step); every window keeps its own
 * damping and accept / reject state.  A window's `converged` flag reports whether some accepted step met
 * rel_cost_tol or some step was rejected at lambda_max (iteration then continues to lm_iters).  autotune != 0 times one LM step of each candidate launch
 * shape (threads per CTA, CTAs per SM, CTAs per window) from the same state, keeps the fastest and caches it per (GPU,
 * precision, size class); the chosen shape is readable with ba_batch_launch_shape(windows[0], ...).
 * reports (n, may be NULL): iters, accepted steps, converged, initial and final cost; ms_total = the graph's
 * device time for the whole batch; ms_window = the window's own time on its CTA.  The instantiated graph is
 * kept with windows[0] (until it is destroyed) and launched again when the same windows, in the same order,
 * are solved with the same iteration count. */
ba_status ba_solve_batch(ba_problem* const* windows, int n, int lm_iters, int autotune, ba_solve_report* reports);
ba_status ba_batch_launch_shape(const ba_problem* p, int* threads, int* grid);
/* CTAs per window (the cluster size) of the last batched solve started from p, and how many of its windows (the
 * largest) ran on clusters; the others ran on single CTAs.  Either pointer may be NULL. */
ba_status ba_batch_ctas_per_window(const ba_problem* p, int* ctas, int* windows_on_clusters);

/* Learned correction of the block-Jacobi preconditioner.  The paper solves the reduced system directly; this
 * optional preconditioner for the PCG solve has no counterpart there.  Per diagonal block b of S (6 wide):
 *   features x_b (32): the 21 upper entries of D_b^-1/2 S_bb D_b^-1/2 (D_b = diag S_bb); over the row's
 *     off-diagonal blocks c, with n_bc = |D_b^-1/2 S_bc D_c^-1/2|_F: log(1+count), sum, max, sum of squares;
 *     the entity type one-hot (camera, plane, VP); zeros.
 *   network: y = W2^T relu(W1^T ((x - mu)/sigma) + b1) + b2, 32 -> 128 -> 21 (BF16 weights at inference).
 *   block: M^ = inv(S^_bb) + sym(y) (no correction in padded or held dimensions), M = D^-1/2 M^ D^-1/2, used
 *     when positive definite, else plain block-Jacobi for that block.
 * Parameter vector (float): mu (32), sigma (32), W1 (32 x 128, row-major by input), b1 (128), W2 (128 x 21,
 * row-major by hidden unit), b2 (21); ba_precond_param_count() values.  Active when options.precond is
 * BA_PRECOND_LEARNED and weights are set. */
int ba_precond_param_count(void);
ba_status ba_precond_set_weights(ba_problem* p, const float* params, int64_t n);
/* Features (na x 32, host) and real-dimension masks (na bytes, bit k = dimension k is real) of the last reduced
 * system built by ba_build_reduced. */
ba_status ba_precond_features(ba_problem* p, float* X, uint8_t* mask);
/* The preconditioner blocks (na x 36, host, row-major 6x6) for the last reduced system: learned when active,
 * else block-Jacobi; *fallbacks receives the number of learned blocks that fell back. */
ba_status ba_precond_blocks(ba_problem* p, double* blocks, int* fallbacks);
/* Training on the GPU (all arrays device memory, FP32).  Samples: X (n x 32), E (n x 21: the upper entries of
 * T^_b - inv(S^_bb), T^_b = D_b^1/2 [inv(S)]_bb D_b^1/2), mask (n).  Loss = mean_b |sym(y_b) - E_b|_F^2 over real
 * dimensions.  ba_mlp_grad: loss and gradient (the trained parameters, i.e. all but mu and sigma, in the
 * parameter order) over all n samples.  ba_precond_train: `steps` Adam steps (Kingma & Ba 2015; beta 0.9 /
 * 0.999, eps 1e-8) on consecutive mini-batches of `batch` samples, starting at step count t0; updates params and
 * the moment vectors adam_m / adam_v in place.  work: device scratch of ba_mlp_work_floats(batch) floats. */
int64_t ba_mlp_work_floats(int64_t batch);
ba_status ba_mlp_grad(int64_t n, const float* X, const float* E, const uint8_t* mask, const float* params,
                      float* grad, double* loss, float* work, void* cuda_stream);
ba_status ba_precond_train(int64_t n, const float* X, const float* E, const uint8_t* mask, float* params,
                           float* adam_m, float* adam_v, int t0, int steps, int64_t batch, float lr, float* work,
                           double* loss_last, void* cuda_stream);

/* Allocation-free PCG (no counterpart in the paper; an addition for embedding the solver).
 *
 * Solves S x = b by the library's block-Jacobi PCG for callers that must not allocate device memory while
 * they run -- for example a solver inside an application whose GPU memory is handed out once by its own
 * arena, or a per-frame loop that is not allowed to call cudaMalloc.  The call performs no cudaMalloc,
 * cudaFree or allocating library routine: every scratch vector lives in one fixed device array inside
 * libba (about 2.3 MB, held by every GPU that loads the library until the process exits).
 *
 *   n_block_rows   block rows of S, each 6 wide, 1 <= n <= 4096
 *   nnz_blocks     stored 6x6 blocks (both triangles), n <= nnz <= 4194304
 *   row_ptr        HOST array (n + 1) of the block-CSR row offsets; every row holds its diagonal block
 *   cols           DEVICE array (nnz) of block column indices
 *   vals           DEVICE array (nnz x 36) of row-major 6x6 blocks, double; S symmetric positive definite
 *   b              DEVICE array (6 n), right-hand side
 *   x              DEVICE array (6 n), output: the PCG iterate when |r_k| <= rel_tol |b| or max_iters is reached
 *   cuda_stream    stream to run on (NULL = default stream); the call returns after the work has finished
 *   iters, rel     optional outputs: PCG iterations and final |r_k| / |b|
 *   err, err_len   optional buffer for a message on failure
 * Returns BA_ERR_ARG (with a message) for sizes beyond the limits above, a missing diagonal block, an
 * out-of-range column or a diagonal block that is not positive definite (no solve is attempted then),
 * BA_ERR_CUDA if a CUDA call fails.
 * The call reads status flags back to the host and synchronises cuda_stream several times, so it cannot be
 * recorded into a CUDA graph: do not call it while a stream of its device is being captured.
 * The first call on a device finds the device address of the scratch array (cudaGetSymbolAddress) with that
 * device current and keeps it for the life of the process; after a cudaDeviceReset of that device in the
 * calling process the kept address is stale, so do not call this entry point again after such a reset.
 * Every call shares the scratch array and leaves the previous call's contents in it (the call initialises
 * everything it reads), so calls whose GPU work overlaps -- from two host threads, or on two streams of one
 * device -- race on it. */
ba_status ba_pcg_solve_static(int64_t n_block_rows, int64_t nnz_blocks, const int32_t* row_ptr,
                              const int32_t* cols, const double* vals, const double* b, double* x,
                              double rel_tol, int max_iters, void* cuda_stream, int* iters, double* rel,
                              char* err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* BA_H */
