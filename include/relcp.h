/*
 * relcp.h -- C ABI of the GB300 ReLCP library.
 *
 * One time step of frictionless contact between smooth, strictly convex rigid
 * bodies (ellipsoids) by recursive constraint augmentation, following
 * "Smooth-Rigid-Body Contact as a ReLCP" (arXiv 2506.14097):
 *
 *   Algorithm 1 (overdamped recursive augmentation time step) and its
 *   inertial variant (Eq. relcp_inertial): build single-constraint
 *   shared-normal signed-distance (SNSD) constraints between near-contacting
 *   pairs, solve the LCP, move to the trial configuration, evaluate the true
 *   SNSD of every candidate pair there, append one frozen-normal, pulled-back
 *   constraint per pair that overlaps by more than eps_NCP (Sec. 3.1.3),
 *   re-solve, and repeat until the geometric stopping rule
 *   max overlap <= eps_NCP (Eq. gap_stopping_rule) holds.
 *
 * Conventions
 *   - Arrays are row-major: x is n x 3, q is n x 4 as (s, w1, w2, w3)
 *     (Hamilton product, R(q) maps body to world), semi-axes n x 3,
 *     velocities and forces n x 6 as (u, omega) / (f, tau), omega and tau in
 *     the world frame (Sec. 2.1.1: C = [.., x, s, w, ..], U = [.., u, omega, ..]).
 *   - Units are the caller's.  A box side of 0 makes that axis open.
 *   - Every call returns relcp_status; nothing throws across the ABI.  On
 *     RELCP_ERR_CUDA / RELCP_ERR_INVALID_ARG a message is available from
 *     relcp_last_error() (per thread, valid until the next failing call).
 *   - Device-side failures (an LCP that hits its iteration cap, a Newton
 *     solve that does not converge, a bounded device wait that gives up) set
 *     a status word that relcp_step reads back and returns; the GPU never
 *     traps and every wait inside the library is bounded.
 *   - Ownership: the caller owns every pointer it passes; inputs are copied.
 *     The context owns all device memory it allocates (stream-ordered, on
 *     the stream given to relcp_create) and frees it in relcp_destroy.
 *   - Pointers marked "ptr_kind" may be host (RELCP_PTR_HOST) or device
 *     (RELCP_PTR_DEVICE) memory; entry points documented as "device" take
 *     device pointers only.
 */
#ifndef RELCP_H
#define RELCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum relcp_status {
    RELCP_OK = 0,
    RELCP_ERR_INVALID_ARG = 1,      /* bad size, NaN, non-unit quaternion, bad enum */
    RELCP_ERR_CUDA = 2,             /* a CUDA runtime call failed */
    RELCP_ERR_CAPACITY = 3,         /* a caller-sized output was too small */
    RELCP_ERR_NOT_CONVERGED = 4,    /* an LCP stopped at lcp_max_iter above lcp_tol */
    RELCP_ERR_RECURSION_LIMIT = 5,  /* overlap remained after max_recursion augmentations */
    RELCP_ERR_NEWTON = 6,           /* an SNSD Newton solve did not converge */
    RELCP_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up */
    RELCP_ERR_STATE = 8             /* call out of order (e.g. step before set_bodies) */
} relcp_status;

/* RELCP_OVERDAMPED_2D: the overdamped law in the z = 0 plane (the growing colony of Sec. 5.4): the
 * generalised velocity has the three components (u_x, u_y, omega_z) with the SPD mobility
 * diag(1/(xi L), 1/(xi L), 12/(xi L^3)) of Eq. ellipsoid_mobility; every row keeps its entries on those
 * components only, U_free is projected onto them, so bodies given in the plane (z = 0, rotations about z)
 * stay in it. */
enum { RELCP_INERTIAL = 0, RELCP_OVERDAMPED = 1, RELCP_OVERDAMPED_2D = 2 };
enum { RELCP_FP64 = 0, RELCP_MIXED = 1 };
enum { RELCP_GUESS_COLD = 0, RELCP_GUESS_MLP = 1 };
enum { RELCP_PTR_HOST = 0, RELCP_PTR_DEVICE = 1 };
/* Body shape of a scene.  RELCP_SHAPE_ELLIPSOID: semi-axes (a, b, c) along the body axes.
 * RELCP_SHAPE_SPHEROCYLINDER (the colony cells of Sec. 5.4): a segment of half-length h along the body x
 * axis swept by a ball of radius rho, given as the semi-axes row (h + rho, rho, rho); its SNSD is the
 * segment distance minus the radii, with the normal along the closest points and the first minimal
 * candidate of (interior stationary point, s = -h_a, s = +h_a, t = -h_b, t = +h_b) taken when parallel
 * segments tie.  Spherocylinders are stepped with the overdamped laws only, take no learned start, and
 * intersecting segments (no normal) report RELCP_ERR_NEWTON. */
enum { RELCP_SHAPE_ELLIPSOID = 0, RELCP_SHAPE_SPHEROCYLINDER = 1 };

/* Time-step parameters (Algorithm 1: Require C^k, F_ext, M, eps_NCP). */
typedef struct relcp_config {
    int32_t dynamics;      /* RELCP_INERTIAL (Eq. law_inertia), RELCP_OVERDAMPED (Eq. law_overdamped) or
                              RELCP_OVERDAMPED_2D (the same law in the z = 0 plane) */
    int32_t precision;     /* RELCP_FP64: every operation FP64.  RELCP_MIXED: FP32 LCP iterations, SNSD
                              Newton iterations and constraint-row assembly; FP64 SNSD polish (Phi),
                              row offsets (Phi + c d^T U), overlap test, LCP residual and the state; the
                              LCP iterations are refined by an FP64 residual (RELCP_FLAG_NO_LCP_REFINE). */
    int32_t guess;         /* SNSD Newton start: RELCP_GUESS_COLD or RELCP_GUESS_MLP (needs relcp_load_mlp).
                              With RELCP_GUESS_MLP the network seeds a step's C^k evaluation when that
                              step evaluates at least 4096 pairs (decided on the device); fewer pairs (the
                              usual case once a step carries the previous step's values) take the cold
                              seeds, whose Newton solves are cheaper than the network's fixed latency.
                              Either start converges to the same SNSD within the Newton tolerance. */
    int32_t lcp_max_iter;  /* projected-gradient iteration cap per LCP (> 0); a refined mixed solve
                              applies it to its FP32 iterations and, apart, to the correction
                              iterations of all its refinement rounds together */
    int32_t max_recursion; /* augmentation cap; 0 gives the single-constraint SNSD-LCP */
    int32_t n_scenes;      /* 1 (batched scenes are a separate entry point) */
    double dt;             /* time step (> 0) */
    double eps_ncp;        /* overlap tolerance eps_NCP (> 0, Eq. gap_stopping_rule) */
    double box[3];         /* periodic box sides at C^k; 0 = open axis */
    double skin;           /* candidate pair: centre distance <= R_i + R_j + skin, R = largest semi-axis */
    double phi_skin;       /* initial constraint set A_0: pairs with Phi(C^k) <= phi_skin */
    double drag_xi;        /* overdamped drag coefficient xi of Eq. ellipsoid_mobility (> 0) */
    double density;        /* inertial: mass density (> 0) */
    double strain_rate;    /* overdamped, fully periodic box only: affine background velocity
                              strain_rate * (x - box/2); the box scales by (1 + strain_rate dt) per step */
    double lcp_tol;        /* LCP stop: max_a |min(A_aa gamma_a, g_a)| <= lcp_tol (distance units) */
    uint64_t seed;         /* reserved for randomised components (MLP training batches) */
    uint32_t fault_inject; /* host-side fault injection mask, RELCP_FAULT_* (tests) */
    uint32_t flags;        /* RELCP_FLAG_* */
    int32_t shape;         /* RELCP_SHAPE_* of every body (batched scenes: of every scene) */
    int32_t reserved;      /* 0 */
} relcp_config;

/* fault injection (host side only; nothing is injected on the GPU) */
enum {
    RELCP_FAULT_ROW_CAPACITY = 1u, /* pretend the row buffer is full: the step reports RELCP_ERR_CAPACITY */
    RELCP_FAULT_LCP_ITERS = 2u,    /* run every LCP with a cap of 1 iteration */
    RELCP_FAULT_LCP_TIMEOUT = 4u,  /* the LCP launch's waits give up after 2 ms, and its last block leaves
                                      before arriving at the first grid barrier: the other blocks' wait runs
                                      out, the launch ends and the step reports RELCP_ERR_TIMEOUT with the
                                      context still usable */
    RELCP_FAULT_NEWTON_ITERS = 8u  /* cap every SNSD Newton phase at 1 iteration: pairs whose start is not
                                      already stationary are not converged and the step reports
                                      RELCP_ERR_NEWTON */
};
enum {
    RELCP_FLAG_PHASE_TIMING = 1u,  /* record per-phase CUDA-event timings in relcp_step_stats */
    RELCP_FLAG_NO_WARM_START = 2u, /* start every LCP_0 from gamma = 0 instead of the previous step's
                                      gamma of the same pair (the solution is the same within lcp_tol) */
    RELCP_FLAG_JACOBI = 4u,        /* projected-gradient steps scaled by 1 / A_aa, BB lengths in the
                                      matching metric (same solution, fewer iterations on uneven rows) */
    RELCP_FLAG_NO_LCP_REFINE = 256u, /* mixed path: solve each LCP by FP32 iterations to lcp_tol directly.  By
                                      default the FP32 iterations hand over once below 10 x lcp_tol (after 8
                                      more iterations) or when they stall (no 10% decrease of the residual in
                                      128 iterations); the residual of that iterate is then taken in FP64 and
                                      the correction solved in FP32, up to eight rounds (iterative refinement:
                                      the FP32 rounding then scales with the correction, not with the contact
                                      forces, and does not stall the solve above lcp_tol) */
    RELCP_FLAG_LEARNED_ALWAYS = 128u, /* with RELCP_GUESS_MLP: run the learned start on every C^k evaluation of
                                      at least one pair (by default it runs when a step evaluates 4,096 pairs
                                      or more at C^k, where its fixed cost pays) */
    RELCP_FLAG_HOST_STAGING = 64u, /* relcp_set_bodies / relcp_get_bodies copy host arrays through pinned
                                      staging buffers even where the device can read and write the caller's
                                      host memory in place (through the host page tables) */
    RELCP_FLAG_GRAPH = 32u,        /* replay the step's first level (broad-phase filter to overlap test, the
                                      LCP launched between the two graphs) from CUDA graphs captured per
                                      configuration; pays off only while the cached pair list is not rebuilt
                                      (every rebuild changes the configuration and costs a new capture) */
    RELCP_FLAG_LCP_TIMING = 16u,   /* CUDA events around the LCP kernel launches only (ms_lcp_kernel,
                                      lcp_alg_bytes), without the per-phase events; an event record costs the
                                      host ~2 us on this hardware */
    RELCP_FLAG_NO_SNSD_REUSE = 8u  /* evaluate the SNSD of every candidate pair at C^k.  By default a
                                      pair that was a candidate in the previous step takes its C^k
                                      values from that step's last overlap test, which evaluated it at
                                      the configuration the step accepted (= this step's C^k); only
                                      new pairs are evaluated */
};

#define RELCP_MAX_DEPTH_STATS 64

/* Diagnostics of the last relcp_step call (its last step when nsteps > 1). */
typedef struct relcp_step_stats {
    int64_t n_bodies;
    int64_t n_pairs;            /* candidate pairs at C^k */
    int64_t n_rows;             /* constraints after the last augmentation */
    int64_t n_rows0;            /* |A_0| */
    int32_t depth;              /* augmentations performed (0 = accepted after the first LCP) */
    int32_t status;             /* relcp_status of the step */
    int32_t lcp_iters_total;
    int32_t newton_iters_max;   /* largest SNSD Newton iteration count of the step */
    int32_t lcp_iters[RELCP_MAX_DEPTH_STATS];        /* per recursion */
    int32_t rows_per_rec[RELCP_MAX_DEPTH_STATS];     /* constraints solved at each recursion */
    double lcp_residual;        /* final LCP residual (FP64) */
    double max_overlap;         /* max_p (-Phi_p)_+ at the accepted configuration (FP64) */
    double box[3];              /* box sides after the step */
    double ms_broadphase, ms_snsd, ms_lcp, ms_augment, ms_total; /* only with RELCP_FLAG_PHASE_TIMING */
    int64_t steps_done;         /* steps since relcp_set_bodies */
    int32_t guess_used;         /* 1 when the learned SNSD guess seeded this step's C^k evaluation */
    int32_t newton_fallbacks;   /* pairs of the learned start whose guess the network itself declined
                                   (trust logit <= 0): their Newton solve started cold */
    /* kernel-level timing: CUDA events around each launch of the persistent LCP
     * kernel (with RELCP_FLAG_PHASE_TIMING or RELCP_FLAG_LCP_TIMING) and of the
     * SNSD kernel (with RELCP_FLAG_PHASE_TIMING) */
    double ms_lcp_kernel;       /* sum over the step's LCP launches */
    double lcp_alg_bytes;       /* algorithmic bytes of those launches: per projected-gradient
                                   iteration 136 B per row + 150 B per body (FP64), 76 B + 75 B (mixed) */
    double ms_snsd_kernel;      /* sum over the step's SNSD launches */
    int64_t snsd_evals;         /* pair evaluations in those launches */
    int32_t lcp_launches;
    int32_t snsd_launches;
    int32_t pair_list_rebuilt;  /* 1 when the cached candidate list was rebuilt in this step */
    int32_t graph_replayed;     /* 1 when the step's first level ran as a replayed CUDA graph */
    int64_t newton_iters_c0;    /* Newton iterations summed over the pairs of the C^k evaluation */
    int64_t snsd_c0_evaluated;  /* pairs evaluated at C^k (the rest reused the previous step's last
                                   overlap test; see RELCP_FLAG_NO_SNSD_REUSE) */
    double host_ms;             /* host time of the step call */
    double host_wait_ms;        /* of which waiting for the device (stream synchronisations) */
} relcp_step_stats;

typedef struct relcp_ctx relcp_ctx;

/* Last error message of the calling thread ("" when none). */
const char* relcp_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts and stateless calls); lets a caller count the launches of a region. */
int64_t relcp_kernel_launches(void);

/* Library and device description (sm_103a build, SM count). */
relcp_status relcp_version(int32_t* major, int32_t* minor, int32_t* sm_count);

/* Create a context on the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = legacy default stream) on which every later call of this context
 * enqueues its work.  *out receives the context. */
relcp_status relcp_create(const relcp_config* cfg, void* cuda_stream, relcp_ctx** out);

/* Replace the configuration (dt, tolerances, box, precision ...).  The body
 * state is kept. */
relcp_status relcp_set_config(relcp_ctx* ctx, const relcp_config* cfg);

/* Load the body state C^k (and U^k, F_ext).  n >= 0.  scene_offsets must be
 * NULL (single scene).  x: n x 3; q: n x 4 (normalised on load; |q| must be
 * within 1e-6 of 1); semi_axes: n x 3 (> 0); vel: n x 6 or NULL (= 0):
 * inertial, the velocity U^k; overdamped, a background velocity added to
 * U = M (F_ext + D gamma); f_ext: n x 6 or NULL (= 0).  dt_per_scene must be
 * NULL.  Periodic positions are wrapped into [0, box).  Resets steps_done.
 * Host arrays are read in place by the device where it can reach pageable
 * host memory through the host page tables (Grace hosts), else through pinned
 * staging (always with RELCP_FLAG_HOST_STAGING); the call returns once the
 * arrays have been read.  An invalid body is reported as "body <i>: <reason>"
 * (the smallest such index) with the context unchanged.  A state equal, bit
 * for bit, to the current one keeps everything the next step carries over;
 * moved bodies keep the cached pair list (its displacement bound still
 * guards it) and the warm starts. */
relcp_status relcp_set_bodies(relcp_ctx* ctx, int64_t n, const int32_t* scene_offsets, const double* x,
                              const double* q, const double* semi_axes, const double* vel,
                              const double* f_ext, const double* dt_per_scene, int32_t ptr_kind);

/* Advance nsteps >= 1 ReLCP time steps (Algorithm 1 per step).  Returns the
 * first non-OK status; the state then holds the configuration accepted by
 * that step (or the last good one for RELCP_ERR_CUDA and RELCP_ERR_TIMEOUT,
 * after which the context stays usable: every device wait is bounded in
 * time).  RELCP_ERR_NOT_CONVERGED (an LCP reached lcp_max_iter),
 * RELCP_ERR_RECURSION_LIMIT (max_recursion augmentations, the last trial
 * accepted) and RELCP_ERR_NEWTON (an SNSD solve did not converge) still accept
 * the step; RELCP_ERR_CAPACITY does not. */
relcp_status relcp_step(relcp_ctx* ctx, int32_t nsteps);

/* Copy out the state: x n x 3 (wrapped), q n x 4, vel n x 6 = velocity of
 * the last step (inertial: U^{k+1}; overdamped: U = U_free + M D gamma).
 * Any pointer may be NULL.  Host arrays are written in place by the device
 * where it reaches pageable host memory, else through pinned staging (as for
 * relcp_set_bodies).  Synchronises the context stream. */
relcp_status relcp_get_bodies(relcp_ctx* ctx, double* x, double* q, double* vel, int32_t ptr_kind);

/* Current periodic box sides (they change under strain_rate). */
relcp_status relcp_get_box(relcp_ctx* ctx, double* box3);

/* Diagnostics of the last step. */
relcp_status relcp_stats(relcp_ctx* ctx, relcp_step_stats* out);

/* Candidate pairs of the last step (at its C^k), i-major with j ascending:
 * pairs cap x 2 int32.  *n_out = number of pairs (RELCP_ERR_CAPACITY when it
 * exceeds cap; nothing is written then).  phi0: SNSD at C^k per pair (cap
 * doubles) or NULL. */
relcp_status relcp_get_pairs(relcp_ctx* ctx, int32_t* pairs, double* phi0, int64_t cap, int64_t* n_out,
                             int32_t ptr_kind);

/* Constraint rows of the last step in creation order (A_0 first, then each
 * augmentation block in pair order).  ids: cap x 4 int32 = (body a, body b,
 * recursion index, candidate-pair index); geom: cap x 11 doubles =
 * (n[3], r_a x n [3], r_b x n [3], offset q, A_aa); gamma: cap doubles (the
 * final LCP solution).  Any pointer may be NULL. */
relcp_status relcp_get_rows(relcp_ctx* ctx, int32_t* ids, double* geom, double* gamma, int64_t cap,
                            int64_t* n_out, int32_t ptr_kind);

/* Contact velocity K D gamma of the last LCP (n x 6; K = M or dt M^-1). */
relcp_status relcp_get_contact_velocity(relcp_ctx* ctx, double* uc, int32_t ptr_kind);

void relcp_destroy(relcp_ctx* ctx);

/* ------------------------------------------------------------------ */
/* Stateless entry points: one hot-path step each, on device pointers,  */
/* enqueued on `stream`.  They allocate their scratch stream-ordered.   */
/* ------------------------------------------------------------------ */

/* Candidate pairs (near-contacting pairs of Algorithm 1's initialisation):
 * all i < j with |min_image(x_j - x_i)|^2 <= (rb_i + rb_j + skin)^2, the
 * squared length summed as ((dx dx + dy dy) + dz dz), every operation
 * rounded separately (decisions are reproducible bit for bit).
 * x: n x 3 device; rb: n device; box3: host (0 = open axis).  pairs: device
 * cap x 2 int32, i-major, j ascending.  *n_out (host) = pair count
 * (RELCP_ERR_CAPACITY when > cap).  Synchronises `stream`. */
relcp_status relcp_broadphase(int64_t n, const double* x, const double* rb, const double* box3, double skin,
                              int32_t* pairs, int64_t cap, int64_t* n_out, void* stream);

/* Shared-normal signed distance (Sec. 2.1.4, n_a = -n_b; y_b - y_a = Phi n)
 * of every listed pair: Phi = max_{|n|=1} n.d - sqrt(n.P_a n) - sqrt(n.P_b n)
 * with P = R diag(a^2) R^T and d the minimum-image c_b - c_a, by damped
 * Newton on the unit sphere.  pairs: npairs x 2 int32 device; x n x 3, q n x 4,
 * axes n x 3 device; box3 host.  out: npairs x 10 device =
 * (Phi, n[3], r_a[3] = y_a - c_a, r_b[3] = y_b - c_b).  iters: npairs int32
 * device or NULL (Newton iterations; negative when not converged).
 * precision: RELCP_FP64 or RELCP_MIXED.  Returns RELCP_ERR_NEWTON if any
 * pair did not converge (outputs still written).  Synchronises `stream`. */
relcp_status relcp_snsd_eval(int64_t npairs, const int32_t* pairs, int64_t n, const double* x, const double* q,
                             const double* axes, const double* box3, int32_t precision, double* out,
                             int32_t* iters, void* stream);

/* Result of one LCP solve. */
typedef struct relcp_lcp_info {
    int32_t iterations;
    int32_t status;       /* relcp_status */
    double residual;      /* max_a |min(A_aa gamma_a, g_a)| at exit (FP64) */
    int32_t grid_blocks;  /* persistent-kernel CTAs used */
    int32_t one_barrier;  /* 1: the iterations ran with one grid barrier each (mixed path with every row
                             in a thread of its own), 0: two grid barriers per iteration */
} relcp_lcp_info;

/* Matrix-free LCP (Eq. cqpp / Lemma LCP <=> CQP): find gamma >= 0 with
 *   g = q + c D^T K D gamma >= 0,  gamma . g = 0,
 * by projected gradient with Barzilai-Borwein steps.  Rows (device):
 * ia, ib: nrows int32 bodies; geom: nrows x 9 doubles (n, r_a x n, r_b x n),
 * the row [-n, -(r_a x n), n, (r_b x n)] on the (u, omega) blocks of a, b;
 * qv: nrows doubles.  K: nbodies x 7 doubles = (k_t, Kr_xx, Kr_yy, Kr_zz,
 * Kr_xy, Kr_xz, Kr_yz): the body operator diag(k_t I, Kr) (K = M overdamped,
 * dt M^-1 inertial).  gamma: nrows doubles, in = warm start (>= 0), out =
 * solution.  uc: nbodies x 6 doubles out = K D gamma.  precision as above.
 * tol: stop when max_a |min(A_aa gamma_a, g_a)| <= tol.  info: host.
 * Synchronises `stream`. */
relcp_status relcp_lcp_solve(int64_t nrows, int64_t nbodies, const int32_t* ia, const int32_t* ib,
                             const double* geom, const double* qv, const double* K, double c,
                             int32_t precision, double tol, int32_t max_iter, double* gamma, double* uc,
                             relcp_lcp_info* info, void* stream);

/* ------------------------------------------------------------------ */
/* Learned SNSD initial guess                                           */
/* ------------------------------------------------------------------ */
/* A small MLP proposes the Newton start of the SNSD solve at C^k; Newton on
 * the sphere decides every result (a bad guess costs iterations,
 * never accuracy).  The paper uses no learned component: this is the learned
 * stand-in for the cold start.  Network: 16 inputs -> 128 -> 128 -> 128 -> 8
 * outputs (5 used), ReLU, BF16 tensor-core kernels with FP32 accumulation.
 * Parameters: one FP32 vector of RELCP_MLP_NPARAMS values, row-major
 * W[out][in]: W1 (128x16), b1, W2 (128x128), b2, W3, b3, W4 (8x128), b4;
 * padded outputs 5..7 must be zero.
 * Features of pair (a, b): d = min-image c_b - c_a in a's frame divided by
 * s = max semi-axis(a) + max semi-axis(b) (3); q_rel = conj(q_a) (x) q_b with
 * non-negative scalar part (4); semi-axes of a (3) and of b (3); the analytic
 * seed normalise((P_a + P_b)^-1 d) in a's frame (3).
 * Outputs: correction from the seed to the shared normal in a's frame, times
 * RELCP_MLP_CORR_SCALE (3), Phi / s, trust logit; the Newton start is
 * normalise(seed + correction / RELCP_MLP_CORR_SCALE) where the logit is
 * positive, the cold start elsewhere.  Training targets: RELCP_MLP_CORR_SCALE
 * times (FP64 SNSD normal in a's frame - seed), and Phi / s. */
#define RELCP_MLP_IN 16
#define RELCP_MLP_HID 128
#define RELCP_MLP_OUT 8
#define RELCP_MLP_NPARAMS (128 * 16 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 8 * 128 + 8)
/* the correction is learned scaled by this factor (outputs of order one stay
 * far above the BF16 resolution of the last layer) */
#define RELCP_MLP_CORR_SCALE 32.0f

/* Features (npairs x 16 float, device) of listed pairs (device, as in
 * relcp_snsd_eval); with snsd_out (npairs x 10 from relcp_snsd_eval) also the
 * training targets (npairs x 4 float: RELCP_MLP_CORR_SCALE x (normal in a's
 * frame minus the seed), Phi / s).  With targets the arithmetic is FP64 (the
 * targets resolve the FP64 SNSD normal); without, FP32 as in the step's own
 * inference (the features agree to FP32 rounding). */
relcp_status relcp_mlp_features(int64_t npairs, const int32_t* pairs, int64_t n, const double* x, const double* q,
                                const double* axes, const double* box3, const double* snsd_out, float* feat,
                                float* targets, void* stream);

/* Network outputs (npairs x 8 float) for features (npairs x 16); params device. */
relcp_status relcp_mlp_forward(int64_t npairs, const float* params, const float* feat, float* out, void* stream);

typedef struct relcp_mlp_train_config {
    float lr;          /* Adam step; 0 = compute the loss and gradients only */
    float beta1, beta2, eps;
    float w_phi;       /* weight of (Phi/s - target)^2 */
    float w_trust;     /* weight of the trust logit's cross-entropy */
    float trust_tol;   /* trust label: squared error of the corrected seed below trust_tol times the
                          squared error of the seed alone (1 = "the correction helps") */
    int32_t step;      /* Adam step counter (>= 1 when lr > 0) */
} relcp_mlp_train_config;

/* One training step on a batch (device): loss = mean over samples of
 * |o[0:3] - t[0:3]|^2 + w_phi (o[3] - t[3])^2 + w_trust BCE(o[4], label);
 * forward and backward on the tensor cores; Adam on params (FP32 master) with
 * moments adam_m, adam_v (NPARAMS each, device).  grad_out (device, NPARAMS)
 * or NULL receives the gradient; *loss_out (host) the batch loss.  Allocates
 * its scratch stream-ordered; synchronises `stream`. */
relcp_status relcp_mlp_train_step(int64_t batch, float* params, float* adam_m, float* adam_v, const float* feat,
                                  const float* targets, const relcp_mlp_train_config* cfg, float* grad_out,
                                  double* loss_out, void* stream);

/* Give a context the parameters (host or device, NPARAMS floats) used when
 * its config has guess = RELCP_GUESS_MLP. */
relcp_status relcp_load_mlp(relcp_ctx* ctx, const float* params, int32_t ptr_kind);

/* ------------------------------------------------------------------ */
/* Batched scenes                                                       */
/* ------------------------------------------------------------------ */

/* Many independent periodic scenes of up to RELCP_BATCH_MAX_BODIES bodies,
 * each stepped by the whole of Algorithm 1 (broad phase, SNSD, A_0, the
 * recursive LCP with the overlap test and augmentation, accept) inside ONE
 * persistent kernel launch per relcp_batch_step call: a CTA takes a scene from
 * a device work queue (largest scenes first) and runs all requested steps of
 * it with CTA barriers only.  The launch is captured in a CUDA graph and
 * replayed.  The block size comes from relcp_batch_autotune (timed on the
 * loaded scenes, cached in a JSON file) or relcp_batch_set_threads.
 *   Dynamics, precision (FP64 or MIXED), drag_xi, density, lcp_max_iter and
 *   max_recursion come from the relcp_config given to relcp_batch_create; box,
 *   dt, eps_ncp, skin, lcp_tol and phi_skin are per scene.  guess and
 *   strain_rate must be RELCP_GUESS_COLD and 0.  Bodies of different scenes
 *   never interact. */
#define RELCP_BATCH_MAX_BODIES 1024
#define RELCP_SCENE_PARAMS 8 /* box x, y, z; dt; eps_ncp; skin; lcp_tol; phi_skin */

typedef struct relcp_batch relcp_batch;

typedef struct {
    int32_t status;       /* relcp_status of the scene (worst over its steps) */
    int32_t status_bits;  /* internal device bits (diagnostics) */
    int32_t steps_done;   /* steps completed since relcp_batch_set_scenes */
    int32_t depth_max;    /* deepest recursion of those steps */
    int32_t lcp_iters;    /* projected-gradient iterations, summed over those steps */
    int32_t n_pairs;      /* candidate pairs of the last step */
    int32_t n_rows;       /* constraint rows of the last step */
    int32_t aug_steps;    /* steps since relcp_batch_set_scenes whose overlap test found a violation
                             (Phi < -eps_ncp at a trial): rows were appended, or the recursion cap
                             stopped the step */
    double max_overlap;   /* largest overlap after the last step */
    double lcp_residual;  /* natural residual of the last LCP */
    double max_overlap_all; /* largest overlap after any step since relcp_batch_set_scenes */
} relcp_scene_stats;

/* Create an empty batch on the current device; the stream as in relcp_create. */
relcp_status relcp_batch_create(const relcp_config* cfg, void* cuda_stream, relcp_batch** out);

/* Load the scenes: scene s owns bodies scene_offsets[s] .. scene_offsets[s+1]-1
 * (0 = offsets[0] <= ... , at most RELCP_BATCH_MAX_BODIES per scene; n = 
 * offsets[n_scenes]).  x, q, semi_axes, vel (NULL = 0), f_ext (NULL = 0) as in
 * relcp_set_bodies, n rows each; scene_params: n_scenes x RELCP_SCENE_PARAMS
 * (box sides > 0 for a periodic axis, 0 for an open one; dt, eps_ncp, lcp_tol
 * > 0; skin, phi_skin >= 0).  Positions are wrapped into the scene's box.
 * Resets the per-scene statistics and warm starts. */
relcp_status relcp_batch_set_scenes(relcp_batch* b, int32_t n_scenes, const int32_t* scene_offsets,
                                    const double* x, const double* q, const double* semi_axes, const double* vel,
                                    const double* f_ext, const double* scene_params, int32_t ptr_kind);

/* Advance every scene by nsteps steps in one launch (synchronises the stream).
 * Returns the worst status over the scenes; a scene that runs out of pair or
 * row capacity (RELCP_ERR_CAPACITY) keeps its last accepted state. */
relcp_status relcp_batch_step(relcp_batch* b, int32_t nsteps);

/* Bodies in the order of relcp_batch_set_scenes (x, q: any may be NULL; vel:
 * n x 6 step velocities). */
relcp_status relcp_batch_get_bodies(relcp_batch* b, double* x, double* q, double* vel, int32_t ptr_kind);

/* Per-scene statistics (host array of n_scenes). */
relcp_status relcp_batch_scene_stats(relcp_batch* b, relcp_scene_stats* out);

/* The last step of one scene (Algorithm 1): its candidate pairs at C^k
 * (pairs: host, n_pairs x 2 int32 body indices local to the scene, i < j,
 * i-major with j ascending) and its constraint rows (row_ids: host, n_rows x 4
 * int32 = body a, body b, recursion index that created the row, index of its
 * pair in the pair list), A_0 first, each recursion's rows after it in pair
 * order.  Either output may be NULL (then only the counts are returned);
 * RELCP_ERR_CAPACITY when a given cap is below the count (the counts are still
 * written).  Before the scene's first step both counts are 0. */
relcp_status relcp_batch_get_scene_contacts(relcp_batch* b, int32_t scene, int32_t* pairs, int64_t pair_cap,
                                            int64_t* n_pairs, int32_t* row_ids, int64_t row_cap, int64_t* n_rows);

/* Time the candidate block sizes (64, 128, 256, 512 threads; a size the kernel
 * cannot run with is skipped) on two steps of the loaded scenes
 * (the scenes' state is restored afterwards) and keep the fastest; the result
 * is the block size.  cache_path (may be NULL): a JSON file of earlier choices, keyed by
 * device, precision and the scenes' size histogram; a hit skips the timing, a
 * miss adds the result.  *threads_out (may be NULL) receives the choice. */
relcp_status relcp_batch_autotune(relcp_batch* b, const char* cache_path, int32_t* threads_out);

/* Fix the block size (a multiple of 32 in [32, 1024]); 0 = untuned default (128 threads). */
relcp_status relcp_batch_set_threads(relcp_batch* b, int32_t threads);

void relcp_batch_destroy(relcp_batch* b);

/* ------------------------------------------------------------------ */
/* Allocation-free variant                                              */
/* ------------------------------------------------------------------ */

/* The paper has no counterpart of this entry point: it is a library
 * convenience.  relcp_snsd_eval_noalloc computes exactly what
 * relcp_snsd_eval computes (same kernels, same arguments, same outputs), but
 * allocates no device memory: its scratch (the per-body shape matrices and the
 * device status word) is a fixed file-scope device array of
 * RELCP_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library holds
 * until the process exits.  It is for callers that cannot call cudaMalloc or
 * cudaMallocAsync: a host framework whose caching allocator has reserved the
 * device memory, a real-time loop where an allocation (which may synchronise
 * the device) is not allowed, or a plugin that may allocate only at start-up.
 *   - n must be <= RELCP_NOALLOC_MAX_BODIES, else RELCP_ERR_CAPACITY with a
 *     message; nothing runs then.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture.
 *   - Every call shares the array, which keeps the last call's contents; the
 *     status word is cleared by each call.  Calls whose work overlaps on the
 *     GPU race on the array: serialise them (one stream, one thread at a time).
 *   - Synchronises `stream`.  Returns RELCP_ERR_NEWTON like relcp_snsd_eval. */
#define RELCP_NOALLOC_MAX_BODIES 65536
#define RELCP_NOALLOC_SCRATCH_BYTES (256 + 48 * RELCP_NOALLOC_MAX_BODIES)
relcp_status relcp_snsd_eval_noalloc(int64_t npairs, const int32_t* pairs, int64_t n, const double* x,
                                     const double* q, const double* axes, const double* box3, int32_t precision,
                                     double* out, int32_t* iters, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RELCP_H */
