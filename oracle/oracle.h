/* FP64 CPU oracle for the batched rigid-body step (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg use this
 * library. It shares no code, header or table with the CUDA library.
 *
 * Every quantity is computed from its plain definition in double precision:
 *   - forward kinematics along the body tree (joint transforms composed root->leaf)
 *   - joint-space inertia M = sum_b J_b^T I_b J_b (+ armature), J_b the spatial body
 *     Jacobian about the world origin (Featherstone, Rigid Body Dynamics Algorithms,
 *     ch. 2 and 6: the composite-rigid-body algorithm computes exactly this sum)
 *   - bias forces sum_b J_b^T (I_b a_b + v_b x* I_b v_b) with qacc = 0 and gravity as
 *     a base acceleration (Newton-Euler equations of each body, RBDA ch. 5)
 *   - plane-sphere/capsule/box and box-box contacts, dense contact Jacobian rows
 *   - the convex soft-contact problem (MuJoCo's published constraint model: solref,
 *     solimp impedance, elliptic friction cone; one-sided joint-limit rows) minimised
 *     to convergence by Newton with exact line search
 *   - PD position actuators, optionally clamped by a DC-motor torque-speed line
 *   - semi-implicit Euler with quaternion integration of free joints
 *   - Philox-4x32-10 (Salmon et al., SC'11) for seeded resets and pushes.
 * The paper (mjlab, arXiv 2601.22074) states none of this math; its Architecture
 * section only fixes the batched-world structure. The adopted readings are listed
 * next to each function in oracle.cpp.
 */
#ifndef B3_ORACLE_H
#define B3_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_desc {
  int32_t nbody, njnt, nu, ngeom;
  const int32_t *body_parent;
  const double *body_pos, *body_quat, *body_mass, *body_ipos, *body_inertia;
  const int32_t *jnt_type, *jnt_body;
  const double *jnt_axis, *jnt_pos, *jnt_armature, *jnt_reset_noise, *qpos_reset;
  const int32_t *act_jnt;
  const double *act_kp, *act_kd;
  const int32_t *geom_type, *geom_body;
  const double *geom_size, *geom_pos, *geom_quat;
  const uint32_t *geom_contype, *geom_conaffinity;
  const double *geom_friction;
  double timestep;
  double gravity[3];
  double solref[2];
  double solimp[5];
  int32_t newton_iterations;
  double newton_tolerance;
  int32_t ls_iterations;
  double pivot_tau;
  int32_t contact_cap;
  int32_t push_period;
  double push_sigma;
  const int32_t *jnt_limited;  /* [njnt] 1: hinge/slide range enforced; NULL: none */
  const double *jnt_range;     /* [njnt][2] lower, upper */
  const double *act_dcmotor;   /* [nu][3] stall torque, no-load speed, torque limit; NULL or
                                  stall torque <= 0: ideal PD */
  int32_t hfield_nrow, hfield_ncol;  /* elevation grid of heightfield geoms (type 4) */
  double hfield_size[2];             /* half extents along the geom's x and y */
  const double *hfield_data;         /* [nrow][ncol] heights (row = y index, col = x index) */
} orc_desc;

/* contact record, 20 doubles: g1 g2 b1 b2 dist pos[3] frame[9] mu f_n f_t (|f_t| unused) */
#define ORC_CON_STRIDE 24

typedef struct orc_model orc_model;

orc_model *orc_model_create(const orc_desc *d, char *err, int errlen);
void orc_model_destroy(orc_model *m);
/* out: nq nv nu nbody ngeom npair ncon_max */
void orc_model_info(const orc_model *m, int32_t *out);
/* pair list [npair][2] (geom1, geom2) */
void orc_model_pairs(const orc_model *m, int32_t *out);

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

void orc_fk(const orc_model *m, const double *qpos, double *xpos, double *xquat,
            double *xmat, double *xipos, double *gxpos, double *gxmat);
void orc_mass_matrix(const orc_model *m, const double *qpos, const double *mass_scale,
                     double *M);
void orc_rne(const orc_model *m, const double *qpos, const double *qvel,
             const double *qacc, int gravity, const double *mass_scale, double *tau);
int orc_ltdl(const orc_model *m, const double *M, double *L, double *D);
void orc_ltdl_solve(const orc_model *m, const double *L, const double *D, double *x);
int orc_collide(const orc_model *m, const double *qpos, double *con, int cap);
/* contact rows: J [3*nc][nv], aref [3nc], R [3nc] (R shared per contact), mu [nc] */
int orc_constraints(const orc_model *m, const double *qpos, const double *qvel,
                    const double *mass_scale, double friction_scale, double *con, int cap,
                    double *J, double *aref, double *R, double *mu);
/* box-box narrow phase of two boxes (centres, row-major rotations, half sizes);
 * axis: chosen separating axis (-1 when separated); minov: smallest overlap over axes */
int orc_box_box(const double *cA, const double *RA, const double *hA, const double *cB, const double *RB,
                const double *hB, double *con, int cap, int32_t *axis, double *minov);
/* joint-limit rows of a state: dof [nl], sign [nl] (+1 lower, -1 upper), dist [nl] (< 0),
 * aref [nl], R [nl]; returns nl (at most cap) */
int orc_limits(const orc_model *m, const double *qpos, const double *qvel, const double *mass_scale,
               int32_t *dof, double *sign, double *dist, double *aref, double *R, int cap);
/* cost and Newton minimiser with nc contacts (rows J [3nc][nv]) and nl one-sided limit
 * rows (Jl [nl][nv], arefl, Dl; NULL when nl = 0); lforce [nl] receives the limit forces */
double orc_cost(int nv, const double *M, const double *a_s, int nc, const double *J,
                const double *aref, const double *D, const double *mu, int nl, const double *Jl,
                const double *arefl, const double *Dl, const double *a);
int orc_newton(int nv, const double *M, const double *a_s, int nc, const double *J,
               const double *aref, const double *D, const double *mu, int nl, const double *Jl,
               const double *arefl, const double *Dl, const double *a_init, double *a, double *force,
               double *lforce, int maxiter);
/* Jacobians of a point p (world coordinates) fixed to body b: Jp [3][nv] maps qvel to
 * the point's velocity, Jr [3][nv] to the body's angular velocity (world frame) */
void orc_body_jacobian(const orc_model *m, const double *qpos, int32_t body, const double *p, double *Jp,
                       double *Jr);
void orc_reset(const orc_model *m, uint64_t seed, int32_t world, double *qpos,
               double *qvel);
/* one env step = push event + nsub substeps. state in/out: qpos qvel qacc.
 * con (optional, cap records) receives the last substep's contacts with forces.
 * stats out: [ncon, newton iterations (sum), status bits] */
int orc_step(const orc_model *m, double *qpos, double *qvel, double *qacc,
             const double *ctrl, double friction_scale, const double *mass_scale,
             const double *kp, const double *kd, int nsub, int64_t step_count,
             uint64_t seed, int32_t world, double *con, int cap, int32_t *stats,
             const double *body_inertia /* [nbody][10] mass, com[3], inertia[6]; NULL: model */);
/* threaded over worlds (std::thread); arrays are [W][n] row-major */
int orc_step_batch(const orc_model *m, int nworld, double *qpos, double *qvel,
                   double *qacc, const double *ctrl, const double *friction_scale,
                   const double *mass_scale, const double *kp, const double *kd, int nsub,
                   const int64_t *step_count, uint64_t seed, const int32_t *world_id,
                   int32_t *stats, int nthreads, const double *body_inertia /* [W][nbody][10] or NULL */);

#ifdef __cplusplus
}
#endif
#endif
