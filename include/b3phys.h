/* b3phys: batched per-world rigid-body physics step for B300 (sm_103a).
 *
 * The step advances thousands of independent simulation instances ("worlds")
 * that share one model, each world with its own state and its own expanded
 * per-world parameters. This is the structure the mjlab paper (arXiv
 * 2601.22074, section "Architecture", MuJoCo Warp paragraph) gives for its
 * physics layer: one data object with a leading world dimension, model fields
 * shared by default and expandable per world for domain randomisation, and the
 * step recorded once as a CUDA graph and replayed. The "Manager-Based API"
 * section's Simulate stage fixes the unit of work: d decimation substeps per
 * environment step. The paper gives no physics equations; the step computes
 * (per world, MuJoCo-style order) forward kinematics, the composite-rigid-body
 * mass matrix and its tree-sparse LDL^T factorisation, recursive Newton-Euler
 * bias forces, PD position actuators, plane-sphere/capsule/box contacts, the
 * contact constraint rows, a Newton solve of the convex soft-contact problem
 * with exact line search, and semi-implicit Euler integration.
 *
 * Conventions common to every call:
 *  - Every function returns a b3p_status: 0 (B3P_OK) or a negative error code.
 *    No call aborts, traps or prints. b3p_last_error() gives a message for the
 *    last failing call on the calling host thread.
 *  - Memory: the caller owns every device buffer. The library allocates no
 *    device memory; b3p_batch_plan says how many bytes one batch needs and the
 *    caller passes that region to b3p_batch_create. Host-side handles
 *    (b3p_model, b3p_batch) are small heap objects freed by their destroy calls.
 *  - Streams: every call that touches the device takes the caller's
 *    cudaStream_t (passed as void*, NULL = legacy default stream) and only
 *    enqueues work on it; nothing synchronises unless stated.
 *  - Per-world numeric faults (NaN/Inf, contact overflow, Newton not
 *    converged, FP64 pivot fallback used) are not call errors: they are
 *    reported in the per-world STATUS bit field.
 *  - Multi-world layout: a batch holds one or more model groups; worlds are
 *    numbered group after group. A per-world field of n values per world is
 *    exchanged as a dense array [W_0][n_0] [W_1][n_1] ... in float32 (or the
 *    stated integer type), group after group.
 */
#ifndef B3PHYS_H
#define B3PHYS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t b3p_status;
enum {
  B3P_OK = 0,
  B3P_ERR_INVALID_ARG = -1,          /* NULL pointer, size or index out of range */
  B3P_ERR_BAD_MODEL = -2,            /* descriptor rejected (message says why) */
  B3P_ERR_WORKSPACE_TOO_SMALL = -3,  /* buffer smaller than b3p_batch_plan's figure */
  B3P_ERR_CUDA = -4,                 /* a CUDA runtime call failed */
  B3P_ERR_GRAPH_STALE = -5,          /* captured graph no longer matches the batch */
  B3P_ERR_TIMEOUT = -6,              /* reserved: no call waits on the device today */
  B3P_ERR_BUSY = -7,                 /* request can never be admitted */
  B3P_ERR_UNSUPPORTED = -8           /* feature the library does not implement (message says which) */
};

/* joint and geom types; bits of the per-world STATUS word */
enum { B3P_JNT_FREE = 0, B3P_JNT_HINGE = 1, B3P_JNT_SLIDE = 2 };
enum { B3P_GEOM_PLANE = 0, B3P_GEOM_SPHERE = 1, B3P_GEOM_CAPSULE = 2, B3P_GEOM_BOX = 3, B3P_GEOM_HFIELD = 4 };
enum {
  B3P_STATUS_NAN = 1,            /* non-finite qpos/qvel: the world stops advancing */
  B3P_STATUS_CONTACT_OVERFLOW = 2,
  B3P_STATUS_NOT_CONVERGED = 4,  /* Newton hit its iteration cap above tolerance */
  B3P_STATUS_FP64_FALLBACK = 8,  /* at least one Hessian was refactored in FP64 */
  B3P_STATUS_BAD_PIVOT = 16,     /* non-positive pivot in the mass matrix */
  B3P_STATUS_IDLE = 32           /* parked serving slot: steps skip the world entirely */
};

/* Model descriptor: flat host arrays (float64), read only during
 * b3p_model_create. Body 0 is the world. Bodies are listed parents first
 * (0 <= body_parent[b] < b for b >= 1). A body carries at most one joint; joints
 * are listed in body order; a free joint's body must be a child of the world.
 * Quaternions are (w, x, y, z). Inertia is about the body's centre of mass, in
 * the body frame, as (Ixx, Iyy, Izz, Ixy, Ixz, Iyz). Geom sizes: sphere (r),
 * capsule (r, half length along local z), box (half sizes); planes use their
 * local z axis as normal. A geom pair collides when
 * (contype1 & conaffinity2) | (contype2 & conaffinity1) is nonzero, the geoms sit
 * on different bodies that are not parent and child (unless the parent is the
 * world), and at least one body moves. Supported pairs: plane-sphere,
 * plane-capsule, plane-box. Actuators are PD position servos on hinge/slide
 * joints, at most one per joint: tau = kp (ctrl - q) - kd qdot.
 * qpos layout: free joint 7 (position, quaternion), hinge/slide 1; qvel: free 6
 * (world linear velocity of the body origin, body-frame angular velocity),
 * hinge/slide 1. */
typedef struct b3p_model_desc {
  int32_t nbody, njnt, nu, ngeom;
  const int32_t *body_parent;       /* [nbody] */
  const double *body_pos;           /* [nbody][3] position in the parent frame at q = 0 */
  const double *body_quat;          /* [nbody][4] orientation in the parent frame */
  const double *body_mass;          /* [nbody] */
  const double *body_ipos;          /* [nbody][3] centre of mass in the body frame */
  const double *body_inertia;       /* [nbody][6] */
  const int32_t *jnt_type;          /* [njnt] B3P_JNT_* */
  const int32_t *jnt_body;          /* [njnt] */
  const double *jnt_axis;           /* [njnt][3] body frame (hinge/slide) */
  const double *jnt_pos;            /* [njnt][3] hinge anchor, body frame */
  const double *jnt_armature;       /* [njnt] rotor inertia added to M's diagonal */
  const double *jnt_reset_noise;    /* [njnt] half-width of the uniform reset noise */
  const double *qpos_reset;         /* [nq] centre of the seeded reset */
  const int32_t *act_jnt;           /* [nu] */
  const double *act_kp, *act_kd;    /* [nu] defaults for the per-world KP/KD fields */
  const int32_t *geom_type;         /* [ngeom] B3P_GEOM_* */
  const int32_t *geom_body;         /* [ngeom] */
  const double *geom_size;          /* [ngeom][3] */
  const double *geom_pos;           /* [ngeom][3] body frame */
  const double *geom_quat;          /* [ngeom][4] body frame */
  const uint32_t *geom_contype, *geom_conaffinity;  /* [ngeom] */
  const double *geom_friction;      /* [ngeom] pair friction = max of the two */
  double timestep;                  /* h, seconds per physics substep */
  double gravity[3];
  double solref[2];                 /* time constant (>= 2h enforced), damping ratio */
  double solimp[5];                 /* dmin, dmax, width, midpoint, power */
  int32_t newton_iterations;        /* cap per substep */
  double newton_tolerance;          /* on |grad| / trace(M) */
  int32_t ls_iterations;            /* cap on line-search evaluations */
  double pivot_tau;                 /* FP64 refactor when an FP32 pivot d_k < tau H_kk */
  int32_t contact_cap;              /* contacts kept per world per substep */
  int32_t push_period;              /* env steps between pushes of the first free body (0 off) */
  double push_sigma;                /* std of the planar push velocity, m/s */
  /* optional (NULL / 0: off) */
  const int32_t *jnt_limited;       /* [njnt] 1: the hinge/slide range is enforced by a
                                       one-sided limit row in the constraint solve (MuJoCo's
                                       joint limit: row e_d (lower) or -e_d (upper) while
                                       violated, margin 0, the contact normal row's impedance,
                                       reference and regulariser with A = (M^-1)_dd) */
  const double *jnt_range;          /* [njnt][2] lower < upper (rad or m) */
  const double *act_dcmotor;        /* [nu][3] DC motor: stall torque ts, no-load speed w0,
                                       torque limit tl; the PD torque is clamped to
                                       [clamp(ts (-1 - w/w0), -tl, 0), clamp(ts (1 - w/w0), 0, tl)]
                                       (section "Components": DC motor with velocity-
                                       dependent saturation); ts <= 0: ideal PD */
  int32_t act_delay;                /* env steps between a target's submission and its use
                                       (0..64); the first act_delay steps after a reset use
                                       the reset pose of the actuated joints (section
                                       "Components": actuation delay) */
  /* heightfield terrain (section "Components": terrain): the elevation grid of every
     B3P_GEOM_HFIELD geom (world body only; geom_size unused). The grid spans
     [-hx, hx] x [-hy, hy] in the geom frame with ncol x nrow samples; each cell splits
     along its (i, j)-(i+1, j+1) diagonal into two triangles; the solid lies below; no
     terrain outside the grid. Spheres and capsule end spheres touch the surface at its
     closest point (or along the normal of the triangle under a centre below it); box
     vertices below the surface give up to 4 contacts (the deepest). */
  int32_t hfield_nrow, hfield_ncol;
  double hfield_size[2];            /* hx, hy */
  const double *hfield_data;        /* [nrow][ncol] heights, row = y index, col = x index */
} b3p_model_desc;

typedef struct b3p_model b3p_model;
typedef struct b3p_batch b3p_batch;

typedef struct b3p_options {
  int32_t warps_per_block;   /* worlds per CTA (one warp each); 0 = default (4); the staged
                                placement takes 1..4 (larger values run as 4) */
  int32_t blocks_per_sm;     /* resident CTAs requested per SM; 0 = as many as fit */
  int32_t write_contacts;    /* 1: each step keeps the last substep's contacts for readback */
  int32_t schedule;          /* 0: static grid-stride order; 1: dynamic queue, heaviest models
                                first (results are identical either way) */
  int32_t working_set;       /* 0: fused launch, each world's working set in shared memory;
                                1: fused launch, working sets in a global region of the
                                batch buffer (cached in L1/L2); 2: staged -- one launch per
                                stage over all worlds (2 + 6 d launches per step, all
                                graph-capturable), working sets in that global region;
                                3: grouped staging -- the same stages, the per-world ones
                                that follow each other in one launch (load and smooth
                                dynamics; integration and the next substep's smooth
                                dynamics), collision and solve separate: 3 d + 1 launches.
                                With schedule 1 the staged placements add one ordering
                                launch per substep and run the solve heaviest first. */
  int32_t history;           /* env steps of (qpos, qvel) each world keeps in a ring buffer of the
                                state region (0: none), read back with b3p_get_history -- the
                                rolling record of recent states the paper's termination manager
                                keeps for replaying a world that went non-finite */
  int32_t lane_solve;        /* 1 (staged placements with schedule 1 only, else INVALID_ARG): the
                                Newton solve of worlds with 1..8 contacts runs one world per
                                lane, 32 worlds per warp, for groups whose Hessian keeps M's
                                tree pattern and that have no joint limits (and fit the
                                device's shared memory); other worlds and groups keep one
                                world per warp. Same minimisation, FP32 rounding differs. */
  int32_t smem_scratch;      /* staged placements. 0: the arrays that no later launch reads
                                (the smooth launches' composite inertias, RNE terms, CRBA
                                temporary and body quaternions; the solve's Newton arrays
                                and its copy of M, M's factor and the motion axes) live in
                                each launch's dynamic shared memory, for each launch whose
                                residency (CTAs per SM) the block does not lower; otherwise
                                in the working set. 1: always in the working set. Results
                                are identical either way. b3p_batch_launch_info reports the
                                choice. */
} b3p_options;

typedef struct b3p_sizes {
  uint64_t total_bytes;      /* size of the one device buffer b3p_batch_create takes */
  uint64_t model_bytes, state_bytes, param_bytes, contact_bytes, scratch_bytes;
  int32_t nworld;            /* sum over groups */
  int32_t smem_bytes_per_world;
} b3p_sizes;

typedef struct b3p_buffers {
  void *base;                /* device pointer, 256-byte aligned */
  uint64_t bytes;
} b3p_buffers;

typedef enum b3p_field {
  B3P_FIELD_QPOS = 0,        /* float32 [W][nq] */
  B3P_FIELD_QVEL = 1,        /* float32 [W][nv] */
  B3P_FIELD_QACC = 2,        /* float32 [W][nv], last substep's acceleration */
  B3P_FIELD_STATUS = 3,      /* uint32  [W] B3P_STATUS_* bits of the last step */
  B3P_FIELD_STATS = 4,       /* int32   [W][4]: contacts in the last substep, Newton
                                iterations and FP64 refactors summed over the last step's
                                substeps, line-search evaluations summed likewise */
  B3P_FIELD_STEP_COUNT = 5   /* int32   [W] env steps taken since reset */
} b3p_field;

typedef enum b3p_param {
  B3P_PARAM_FRICTION_SCALE = 0,  /* float32 [W]: multiplies every pair friction */
  B3P_PARAM_MASS_SCALE = 1,      /* float32 [W][nbody]: scales mass and inertia */
  B3P_PARAM_KP = 2,              /* float32 [W][nu] */
  B3P_PARAM_KD = 3,              /* float32 [W][nu] */
  B3P_PARAM_BODY_INERTIA = 4     /* float32 [W][nbody][10]: mass, centre of mass (3, body frame),
                                    inertia about it (Ixx Iyy Izz Ixy Ixz Iyz, body frame);
                                    starts at the model's values; the mass scale multiplies it */
} b3p_param;

/* contact record readback: B3P_CON_FLOATS floats per slot, W x ncon_max slots:
 * geom1 geom2 body1 body2 dist pos[3] frame[9] (normal, tangent1, tangent2 rows)
 * mu force[3] (normal, tangent1, tangent2) force_world[3] (on body2, from body1) */
#define B3P_CON_FLOATS 24

/* last error message of the calling host thread ("" if none) */
const char *b3p_last_error(void);
/* library version string */
const char *b3p_version(void);

/* Copy and validate a descriptor; derive dof layout, tree-sparse mass-matrix
 * pattern, tree levels and collision pairs. Host only. Errors: INVALID_ARG,
 * BAD_MODEL. *out is owned by the caller (b3p_model_destroy). */
b3p_status b3p_model_create(const b3p_model_desc *desc, b3p_model **out);
void b3p_model_destroy(b3p_model *m);
/* out[8] = nq nv nu nbody ngeom npair ncon_max nM (stored mass-matrix entries) */
b3p_status b3p_model_info(const b3p_model *m, int32_t *out);

/* Bytes needed for a batch of nmodels groups with nworld[g] worlds each. Host
 * only. opt may be NULL (defaults). */
b3p_status b3p_batch_plan(const b3p_model *const *models, const int32_t *nworld, int32_t nmodels,
                          const b3p_options *opt, b3p_sizes *out);
/* Lay the batch out in the caller's device buffer (bufs->bytes >= plan
 * total_bytes, else WORKSPACE_TOO_SMALL), upload the models, set every
 * per-world parameter to the model default, zero the state. Enqueues copies on
 * `stream` and waits for them. The models must outlive the batch. Call
 * b3p_reset before the first step. */
b3p_status b3p_batch_create(const b3p_model *const *models, const int32_t *nworld, int32_t nmodels,
                            const b3p_options *opt, const b3p_buffers *bufs, void *stream,
                            b3p_batch **out);
void b3p_batch_destroy(b3p_batch *b);
/* out[4 + 2 * ngroup] (cap entries at most): nworld ngroup, total floats of a
 * QPOS readback, of a QVEL readback, then per group (world_start, nworld) */
b3p_status b3p_batch_info(const b3p_batch *b, int32_t *out, int32_t cap);
/* out[5] (cap >= 5): the launch shape the batch settled on -- worlds (warps) per CTA, the
 * fused launch's grid, then the dynamic shared memory per CTA in bytes of the grouped smooth
 * launches' scratch block, of the solve launch's block and of the lane solve (0: not used). */
b3p_status b3p_batch_launch_info(const b3p_batch *b, int32_t *out, int32_t cap);

/* Seeded reset of worlds world_ids_dev[0..n) (device int32 global world
 * indices), or of every world when world_ids_dev is NULL. qpos = qpos_reset +
 * noise_j (2u - 1) on hinge/slide joints, u = the (j mod 4)-th word of
 * Philox-4x32-10(counter {j / 4, rng_id, 1, 0}, key = seed) mapped to [0, 1)
 * with its top 24 bits; qvel = qacc = 0; step count, status and stats cleared.
 * rng_id = the world's index within its group unless rng_ids_dev (device
 * int32, parallel to world_ids_dev, or to all worlds) gives it. */
b3p_status b3p_reset(b3p_batch *b, uint64_t seed, const int32_t *world_ids_dev,
                     const int32_t *rng_ids_dev, int32_t n, void *stream);

/* Overwrite one per-world parameter of group `group` from a device array
 * (layout in b3p_param). */
b3p_status b3p_set_world_param(b3p_batch *b, int32_t group, b3p_param field, const float *src_dev,
                               void *stream);

/* One environment step of every world: the push event (if due: step count a
 * positive multiple of push_period; velocity kick sigma * Box-Muller of words 0,
 * 1 of Philox(counter {0, rng_id, 2, step count}, key = seed) on the first two
 * dofs of joint 0 when it is free), then `decimation` physics substeps with the
 * PD targets ctrl_dev (float32, dense [W_g][nu_g] per group, group after group;
 * NULL when no group has actuators). The batch's placement decides the launches:
 * one persistent launch with the world state on chip between substeps
 * (working_set 0 or 1), or launches per stage over all worlds (working_set 2: 2 + 6 d
 * launches; 3: 3 d + 1). Results agree up to rounding across placements. */
b3p_status b3p_step(b3p_batch *b, const float *ctrl_dev, int32_t decimation, void *stream);

/* Record nsteps consecutive b3p_step launches as one CUDA graph; step s reads
 * ctrl from ctrl_base_dev + s * ctrl_stride_floats. b3p_graph_launch replays it.
 * A graph goes stale when the batch options change (GRAPH_STALE). */
b3p_status b3p_step_capture(b3p_batch *b, const float *ctrl_base_dev, int64_t ctrl_stride_floats,
                            int32_t decimation, int32_t nsteps, void *stream);
b3p_status b3p_graph_launch(b3p_batch *b, void *stream);

/* Step without any workspace from the caller. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code that is
 * handed a fixed set of input and output buffers by a host framework owning all
 * device memory, or a process whose device memory is fixed when it starts -- and
 * so cannot provide the FP64 pivot-fallback workspace that b3p_step takes from the
 * batch buffer. Here that workspace is a fixed array inside the library,
 * B3P_STATIC_SCRATCH_DOUBLES doubles (32 MiB), which every GPU that loads the
 * library keeps until the process exits; this call allocates nothing and never
 * touches the batch buffer's workspace region. Results match b3p_step's up to
 * floating-point rounding (the two kernels are compiled separately).
 *  - The batch must keep its working sets in shared memory (working_set = 0),
 *    else B3P_ERR_UNSUPPORTED.
 *  - A batch needing more than the array is rejected with B3P_ERR_INVALID_ARG and a
 *    message giving both sizes. A world needs nM + nv doubles when its model keeps
 *    M's tree sparsity in the Newton Hessian, and nv * (nv + 1) when contacts join two
 *    kinematic trees (dense Hessian, e.g. a gripper and a free object); the batch
 *    needs the sum over its groups of W_g times that (nM, nv from b3p_model_info).
 *  - The batch's schedule option is ignored: worlds are taken in index order.
 *  - The first call on a device looks up the array's device address with that
 *    device current (once per device); make that first call before any stream
 *    capture.
 *  - Every call, on every stream and batch, shares the one array, and the array
 *    keeps whatever the last call left in it: the kernel writes each world's slice
 *    completely before reading it, so nothing needs clearing, but two calls that
 *    overlap on the GPU race on it. Serialise them (one stream, or events). */
#define B3P_STATIC_SCRATCH_DOUBLES 4194304
b3p_status b3p_step_static_scratch(b3p_batch *b, const float *ctrl_dev, int32_t decimation, void *stream);

/* Plain comparator: the same step as separate per-stage kernels (load, then per
 * substep kinematics / dynamics / mass matrix / collision / Newton / integration,
 * then store), one model group per launch sequence, the per-world working set in
 * a caller-provided global workspace of b3p_plain_workspace_bytes() bytes (256-byte
 * aligned), no CUDA graph. Same results as b3p_step up to floating-point rounding. */
size_t b3p_plain_workspace_bytes(const b3p_batch *b);
b3p_status b3p_step_plain(b3p_batch *b, const float *ctrl_dev, int32_t decimation, void *workspace_dev,
                          size_t bytes, void *stream);

/* One staged step (batch created with working_set = 2 or 3; a grouped batch is timed
 * through the ungrouped stage launches, which run the same per-stage code) with a CUDA
 * event recorded
 * on the stream before each of its 2 + 6 d launches and after the last; waits for
 * the stream, then ADDS each stage's summed kernel time in milliseconds to
 * stage_ms_host[B3P_NSTAGES] (index = stage: 0 load, 1 kinematics, 2 bias and
 * actuators, 3 mass matrix and smooth solve, 4 collision and contact rows, 5 Newton
 * solve, 6 integration, 7 store) and the launches per stage to launches_host
 * [B3P_NSTAGES] (may be NULL). Same state update as b3p_step. Not capturable (it
 * synchronises); for measurement only. UNSUPPORTED for the fused placements, whose
 * step is a single kernel. */
#define B3P_NSTAGES 8
b3p_status b3p_step_profile(b3p_batch *b, const float *ctrl_dev, int32_t decimation, float *stage_ms_host,
                            int32_t *launches_host, void *stream);

/* Measured FP32 FMA throughput of the current device, the ALU roof of the step's
 * roofline (the step is FP32 arithmetic bound by dependent latency, not a dense
 * contraction or an HBM stream). Launches a probe kernel on every SM at full occupancy:
 * each thread runs eight independent FMA chains, nothing is read from memory. Writes
 * the best of `reps` event-timed launches in FLOP/s (2 per FMA) to *flops_per_s_host and
 * the device's SM count to *sm_count_host. Synchronises the stream; measurement only,
 * not capturable. INVALID_ARG for null outputs or reps < 1, CUDA on a launch error. */
b3p_status b3p_fp32_peak(int32_t reps, double *flops_per_s_host, int32_t *sm_count_host, void *stream);

/* Device-to-device copies of one state field to / from dense caller arrays
 * (layout in b3p_field; bytes must equal the field's size; a batch without worlds takes
 * bytes = 0 and any pointer). */
b3p_status b3p_get_state(b3p_batch *b, b3p_field f, void *dst_dev, size_t bytes, void *stream);
b3p_status b3p_set_state(b3p_batch *b, b3p_field f, const void *src_dev, size_t bytes, void *stream);

/* Contacts of the last substep of the last step (batch created with
 * write_contacts = 1, else UNSUPPORTED): dst_dev receives
 * [sum_g W_g * ncon_max_g][B3P_CON_FLOATS] floats (slots beyond a world's count
 * are stale), count_dev [W] int32. */
b3p_status b3p_get_contacts(b3p_batch *b, float *dst_dev, size_t bytes, int32_t *count_dev,
                            void *stream);

/* Serving primitives (continuous batching of rollout requests over one batch of
 * slots; section "Architecture" keeps all world state on the device between
 * steps, and requests of different morphologies share one launch).
 *  b3p_set_idle: set (idle = 1) or clear the B3P_STATUS_IDLE bit of the listed
 *    worlds (device int32 global indices; NULL = all). Idle worlds cost a status
 *    read per step. b3p_reset clears the bit.
 *  b3p_sample_targets: for every non-idle world, PD targets = reset pose +
 *    sigma_g N(0, 1), the normals drawn by Box-Muller from
 *    Philox-4x32-10(counter {u / 2, rng_id, 3, step count}, key = the world's reset
 *    seed) (cosine for even actuator index u, sine for odd), sigma_dev a device
 *    float32 [ngroup]; written into ctrl_dev in b3p_step's layout. A request's
 *    targets therefore depend only on its seed and its worlds' indices within it.
 *  b3p_gather_state: rows of qpos/qvel/qacc of the listed worlds of one group
 *    (device int32 local indices) packed densely into dst_dev [n][width]. */
b3p_status b3p_set_idle(b3p_batch *b, const int32_t *world_ids_dev, int32_t n, int32_t idle, void *stream);
b3p_status b3p_sample_targets(b3p_batch *b, const float *sigma_dev, float *ctrl_dev, void *stream);
b3p_status b3p_gather_state(b3p_batch *b, int32_t group, b3p_field f, const int32_t *local_ids_dev,
                            int32_t n, float *dst_dev, void *stream);

/* Rollout server (section "Architecture": all world state stays on the device
 * between steps; requests of different morphologies share the same launches).
 * A server owns one batch of world slots per morphology, sized from an HBM budget
 * (the bytes b3p_batch_plan charges per world, the budget split evenly over the
 * morphologies, capped by max_worlds_per_model), plus its device buffers and a
 * pinned host pool for results; it is the one object of this library that
 * allocates device memory itself (at create; none per tick). Requests
 * (morphology, worlds, horizon in env steps, seed) are admitted in arrival order
 * wherever their worlds fit (first fit, lowest free slots), reset from the
 * request seed with rng ids 0..nworld-1, and advanced one env step per tick
 * together with every other active request: targets from b3p_sample_targets
 * (sigma per morphology), then b3p_step. A request that reaches its horizon is
 * retired in the same tick: its final qpos/qvel rows are gathered on the device
 * and copied to pinned host memory behind a CUDA event; its slots are idled and
 * free for the next tick. A result therefore depends only on the request's
 * morphology, seed and horizon, never on its slots or its neighbours.
 *  run_thread = 1: a server thread ticks while requests are queued or active
 *    (b3p_server_tick is then refused); 0: the caller ticks.
 *  b3p_server_submit: BUSY when nworld exceeds the morphology's slot pool (it
 *    could never be admitted), INVALID_ARG for a bad morphology index, nworld < 1
 *    or horizon < 1. Thread-safe.
 *  b3p_server_poll: non-blocking; moves up to max finished results into out. The
 *    host arrays stay valid until b3p_server_release(id). Thread-safe.
 *  A CUDA error inside a tick stops the server: every later call returns it.
 *  Times are seconds on the server's steady clock since b3p_server_create. */
typedef struct b3p_server b3p_server;
typedef struct b3p_server_cfg {
  int32_t nmodels;
  const b3p_model *const *models;   /* outlive the server */
  double hbm_budget_bytes;
  int32_t max_worlds_per_model;     /* 0 = only the budget limits the pools */
  int32_t decimation;
  const float *sigma_host;          /* [nmodels] PD-target std per morphology */
  b3p_options options;              /* placement of the slot batch */
  int32_t max_inflight_ticks;       /* ticks the host may run ahead of the GPU (>= 1) */
  int32_t run_thread;
  int32_t device;                   /* CUDA device of the server */
} b3p_server_cfg;
typedef struct b3p_request {
  int32_t model, nworld, horizon;
  uint64_t seed;
} b3p_request;
typedef struct b3p_result {
  int64_t id;
  int32_t model, nworld;
  const float *qpos;                /* host [nworld][nq], pinned */
  const float *qvel;                /* host [nworld][nv], pinned */
  double t_submit, t_admit, t_done; /* t_done: when a poll saw the copy complete */
} b3p_result;
typedef struct b3p_server_stats {
  int64_t ticks, world_steps, submitted, completed;
  int32_t queued, active, pending;  /* waiting, running, retired but not yet polled */
  int32_t reserved;
} b3p_server_stats;
b3p_status b3p_server_create(const b3p_server_cfg *cfg, b3p_server **out);
void b3p_server_destroy(b3p_server *s);
b3p_status b3p_server_capacity(const b3p_server *s, int32_t *slots, int32_t cap);
b3p_status b3p_server_submit(b3p_server *s, const b3p_request *r, int64_t *id);
b3p_status b3p_server_tick(b3p_server *s, int32_t *active_worlds);
b3p_status b3p_server_poll(b3p_server *s, b3p_result *out, int32_t max, int32_t *n);
b3p_status b3p_server_release(b3p_server *s, int64_t id);
b3p_status b3p_server_get_stats(b3p_server *s, b3p_server_stats *out);
double b3p_server_now(const b3p_server *s);

/* Post-step readouts on the device, so a learning loop never copies state to the host
 * (section "Manager-Based API": the Observe stage after Simulate; section "Components":
 * contact sensor with air time).
 *  b3p_observe: per world of group `group`, the velocity-task observation terms in this
 *    order: gravity direction in the base frame (3), base linear velocity in the base
 *    frame (3), base angular velocity in the base frame (3) -- the base is joint 0 when
 *    it is free, else these 9 are 0 --, then for every hinge/slide joint in joint order
 *    q - q_reset, then their velocities, then the ctrl_dev targets of the group (nu; 0
 *    when ctrl_dev is NULL). out_dev: float32 [W_g][b3p_observe_width]. The gravity
 *    direction is gravity / |gravity| ((0, 0, -1) without gravity).
 *  b3p_contact_sensor: for n bodies (body_ids_dev, device int32) of group `group`, per
 *    world: the net contact force on the body in world coordinates (force_dev [W_g][n][3],
 *    the last substep's contacts: +F on body 2 of a contact, -F on body 1), and the
 *    air-time state state_dev [W_g][n][4] = (in contact, current air time, current
 *    contact time, last air time), owned by the caller (zero it at reset) and advanced
 *    by dt: in contact when |force| > threshold; at touchdown last air time <- current
 *    air time and current air time <- 0; at lift-off current contact time <- 0. Needs a
 *    batch created with write_contacts = 1 (else UNSUPPORTED). */
int32_t b3p_observe_width(const b3p_batch *b, int32_t group);
b3p_status b3p_observe(b3p_batch *b, int32_t group, const float *ctrl_dev, float *out_dev, void *stream);
b3p_status b3p_contact_sensor(b3p_batch *b, int32_t group, const int32_t *body_ids_dev, int32_t n, float threshold,
                              float dt, float *state_dev, float *force_dev, void *stream);
/* The contact sensor with its force history (section "Components": contact sensor with
 * air-time and force-history bookkeeping): as b3p_contact_sensor, and each body's force is
 * also written into a ring of `depth` env steps, history_dev [W_g][n][depth][3] (owned by
 * the caller), slot (step count - 1) mod depth of the world -- the env step the contacts
 * come from (step count counts env steps since the world's reset). Reading the ring from
 * slot (step count mod depth) onwards gives the forces oldest first. depth >= 1. */
b3p_status b3p_contact_sensor_history(b3p_batch *b, int32_t group, const int32_t *body_ids_dev, int32_t n,
                                      float threshold, float dt, float *state_dev, float *force_dev,
                                      float *history_dev, int32_t depth, void *stream);

/* Fused per-world reward and termination of the velocity-tracking task (section
 * "Manager-Based API": the reward manager's weighted sum of terms scaled by the control
 * timestep, with per-term episodic sums and per-term detection of non-finite values; the
 * termination manager's stop conditions -- illegal contacts, time-out, NaN/Inf state;
 * section "Tasks": velocity tracking with penalties on body angular velocity, action rate,
 * joint-limit violation and foot slip). One warp per world of group `group` (forward
 * kinematics and motion axes of the current qpos in shared memory, for the foot
 * velocities). Terms, in this order (raw values; base = joint 0 when it is a free joint,
 * else terms 0-3 and 8 are 0 and the base checks are off; base-frame quantities are the
 * transpose of the base rotation applied to world vectors):
 *   0 exp(-|v_xy - cmd_xy|^2 / sigma_lin^2)   base-frame linear velocity vs command
 *   1 exp(-(w_z - cmd_wz)^2 / sigma_ang^2)    base-frame yaw rate vs command
 *   2 v_z^2                                   base-frame vertical velocity
 *   3 w_x^2 + w_y^2                           base-frame roll/pitch rates
 *   4 sum_u (a_u - a_prev_u)^2                action rate (the group's targets)
 *   5 sum over limited joints of max(0, lo - q) + max(0, q - hi)
 *   6 sum_feet in-contact x |v_foot,xy|^2     world-frame velocity of the foot body origin
 *   7 sum_feet touchdown x (last air time - air_time_target); touchdown = in contact with
 *     contact time <= 1.5 dt (the sensor state advanced by dt this env step)
 *   8 g_x^2 + g_y^2                           gravity direction in the base frame
 *   9 sum of qacc^2 over the dofs of non-free joints
 * Each term contributes weight[k] x raw x dt to reward_dev [W_g]; terms_dev [W_g][10]
 * receives those contributions and episode_dev [W_g][10] accumulates them (the caller
 * zeroes a world's row at its reset). A non-finite contribution is left out of the sum,
 * written as 0, and flagged. done_dev [W_g] (uint32 bits): 1 terminated (any of 4, 8, 16,
 * 32), 2 time-out (step count >= max_episode_steps > 0), 4 non-finite state (qpos, qvel,
 * qacc, or the NaN status), 8 base height below min_base_height (> 0 to enable), 16 base
 * up axis leaning more than max_tilt radians from world up (> 0 to enable), 32 a contact
 * involving a body of illegal_host (needs write_contacts = 1 when nillegal > 0, else
 * UNSUPPORTED), 256 << k term k non-finite. cmd_dev [W_g][3] (vx, vy, wz); action_dev and
 * prev_action_dev are targets in b3p_step's layout (the group's slice is read; NULL when
 * the group has no actuators); sensor_state_dev [W_g][nfeet][4] is the air-time state of
 * b3p_contact_sensor for the feet in feet_host order (needed when nfeet > 0). Device
 * pointers except the body lists; INVALID_ARG for a null required pointer, a body index
 * out of range, more than B3P_REWARD_MAXBODIES bodies in a list or dt <= 0. feet_host and illegal_host are host arrays of at most B3P_REWARD_MAXBODIES
 * bodies each, copied into the launch (the call reads no device memory on the host and
 * does not synchronise, so it can be recorded in a CUDA graph with the step). */
#define B3P_REWARD_NTERMS 10
#define B3P_REWARD_MAXBODIES 16
typedef struct b3p_reward_cfg {
  float weight[B3P_REWARD_NTERMS];
  float sigma_lin, sigma_ang;      /* tracking widths (m/s, rad/s), > 0 */
  float air_time_target;           /* seconds */
  float dt;                        /* control timestep: timestep x decimation */
  float min_base_height;           /* metres; <= 0: off */
  float max_tilt;                  /* radians; <= 0: off */
  int32_t max_episode_steps;       /* env steps; <= 0: no time-out */
  int32_t nfeet;
  const int32_t *feet_host;        /* [nfeet] foot bodies, the sensor's order (host) */
  int32_t nillegal;
  const int32_t *illegal_host;     /* [nillegal] bodies whose contacts terminate (host) */
} b3p_reward_cfg;
b3p_status b3p_reward(b3p_batch *b, int32_t group, const b3p_reward_cfg *cfg, const float *cmd_dev,
                      const float *action_dev, const float *prev_action_dev, const float *sensor_state_dev,
                      float *reward_dev, float *terms_dev, float *episode_dev, uint32_t *done_dev, void *stream);

/* Differential inverse kinematics by damped least squares (section "Manager-Based API":
 * the action manager's differential-IK term): per world of group `group`, from the
 * current qpos, the point p = body origin + R_body offset_host (body frame, 3 floats),
 * its Jacobian J over the group's actuated joints (3 rows, or 6 with the body's angular
 * Jacobian when target_quat_dev is given), e = target_pos - p (and the rotation vector of
 * target_quat (x) body_quat^-1, world frame), and
 *     dq = J^T (J J^T + lambda^2 I)^-1 e,
 * written as PD targets q_a + dq into the group's slice of ctrl_dev (b3p_step's layout;
 * other groups untouched). target_pos_dev [W_g][3], target_quat_dev [W_g][4] (w, x, y, z)
 * or NULL; lambda > 0. Uses one warp and the model's per-world working set in shared
 * memory per world. */
b3p_status b3p_diffik(b3p_batch *b, int32_t group, int32_t body, const float *offset_host,
                      const float *target_pos_dev, const float *target_quat_dev, float lambda, float *ctrl_dev,
                      void *stream);

/* Ray-cast sensor (section "Components": ray-cast sensor, grid or pinhole pattern,
 * distance per ray): per world of group `group`, nray rays fixed to body `body` --
 * origins_dev [nray][3] and unit directions_dev [nray][3] in the body frame (device
 * float32) -- cast from the current qpos against the group's geoms: the world's geoms
 * only when world_only = 1, else every geom not attached to `body`. dist_dev [W_g][nray]
 * receives the distance to the first surface along each ray (0 for an origin inside a
 * solid; max_dist when nothing is hit within max_dist). Planes are half-spaces (solid
 * below), capsules are segments swept by a sphere, boxes are slabs, heightfields are their
 * triangle surfaces walked cell by cell along the ray's ground track. Each world's geom
 * poses come from forward kinematics in shared memory; rays test every geom (no BVH:
 * models hold at most a few dozen primitives). */
b3p_status b3p_raycast(b3p_batch *b, int32_t group, int32_t body, int32_t nray, const float *origins_dev,
                       const float *directions_dev, float max_dist, int32_t world_only, float *dist_dev,
                       void *stream);
/* The ray-cast sensor with hit positions and surface normals (section "Components": a
 * BVH-accelerated ray-cast sensor returning per-ray distances, hit positions and surface
 * normals). As b3p_raycast, plus pos_dev [W_g][nray][3] (origin + distance x direction,
 * world frame; the point at max_dist for a miss) and normal_dev [W_g][nray][3] (outward
 * unit normal of the solid hit, world frame: the plane's z axis, from the sphere centre
 * or the capsule's segment, the box face whose slab the ray enters last, the hit
 * triangle's upward normal; zero for a miss or an origin inside a solid; among geoms hit
 * at the same distance the lowest geom index gives it); either may be NULL. flags: 1 =
 * world geoms only (as world_only); 2 = test every geom in turn instead of the bounding-
 * volume hierarchy (the hierarchy: the kinematic tree, each body's box bounding its geoms
 * and each node's box its subtree, refitted from the current poses on every call; a ray
 * visits only subtrees whose box it enters before its nearest hit so far; the world
 * body's geoms are always tested directly). The results of the two are the same. */
b3p_status b3p_raycast_hits(b3p_batch *b, int32_t group, int32_t body, int32_t nray, const float *origins_dev,
                            const float *directions_dev, float max_dist, int32_t flags, float *dist_dev,
                            float *pos_dev, float *normal_dev, void *stream);

/* The history ring of world `world` (local index) of group `group` in chronological
 * order: dst_dev [history][nq + nv] float32 (qpos then qvel after each of the last
 * min(step count, history) env steps, oldest first; later rows zero) and the number of
 * valid rows in count_dev (device int32). UNSUPPORTED when the batch keeps no history. */
b3p_status b3p_get_history(b3p_batch *b, int32_t group, int32_t world, float *dst_dev, int32_t *count_dev,
                           void *stream);

/* Raw copy of the whole per-world state (qpos, qvel, qacc, counters, seeds,
 * status) for checkpoint / resume; b3p_state_bytes gives the size. */
size_t b3p_state_bytes(const b3p_batch *b);
b3p_status b3p_state_save(b3p_batch *b, void *dst_dev, size_t bytes, void *stream);
b3p_status b3p_state_restore(b3p_batch *b, const void *src_dev, size_t bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* B3PHYS_H */
