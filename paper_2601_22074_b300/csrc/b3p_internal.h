// Internal layout shared by the host library (b3p_host.cpp) and the kernels
// (b3p_step.cu). Not part of the public ABI.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define B3P_HD __host__ __device__
#else
#define B3P_HD
#endif

#define B3P_MAXCHAIN 32   // dofs on any root-to-leaf chain (local arrays, pair decoding)
#ifndef B3P_SMOOTH_AUX
#define B3P_SMOOTH_AUX 1  // grouped staging keeps launch-local scratch in shared memory
#endif
#ifndef B3P_SOLVE_AUX
#define B3P_SOLVE_AUX 1   // staged solve launches keep the Newton arrays in shared memory
#endif
#ifndef B3P_SOLVE_STAGE_INPUTS
#define B3P_SOLVE_STAGE_INPUTS 1   // ... and a copy of M, M's factor and the motion axes
#endif
#define B3P_MAXGROUP 16
#define B3P_PURPOSE_RESET 1u
#define B3P_PURPOSE_PUSH 2u
#define B3P_MAX_DEVICES 64
#ifndef B3P_STATIC_SCRATCH_DOUBLES
#define B3P_STATIC_SCRATCH_DOUBLES 4194304
#endif

// Per-model constants in device memory. Index arrays are int32, real arrays
// float32; every pointer points into the batch buffer.
struct DModel {
  int nb, nj, nu, ng, nq, nv, npair, ncon_max, nM, maxlevel;
  int nq_pad, nv_pad, nu_pad, nb_pad;  // row strides of per-world arrays (multiples of 4)
  int first_free_dof;                  // dof address of joint 0 when it is free, else -1
  int newton_iter, ls_iter, push_period;
  float h, grav[3], ref_b, ref_k, imp[5], tol, pivot_tau, push_sigma;
  int dense;                           // 1: H is a dense nv x nv matrix (cross-tree contacts)
  int maxchain;                        // longest root-to-leaf dof chain (max dof_rowlen)
  int scratch_doubles;                 // FP64 pivot-fallback workspace per world
  int smem_floats;                     // per-world shared-memory footprint (floats)
  // shared-memory offsets (floats) of the per-world arrays
  int o_qpos, o_qvel, o_qacc, o_qs, o_frc, o_ctrl, o_kp, o_kd, o_ms;
  int o_xpos, o_xquat, o_xmat, o_cdof, o_tmp6, o_cvel, o_union;
  int o_M, o_L, o_H, o_Hdiag, o_Ma, o_Mp, o_g, o_p;
  int o_con, o_coni, o_misc, o_lim;
  // joint limits, DC motors, actuation delay
  int nlim, dcmotor, act_delay;
  const int *lim_dof, *lim_qadr;       // [nlim] limited joints' dof and qpos addresses
  const float *lim_range;              // [nlim][2]
  const float *act_dcm;                // [nu][3] stall torque, no-load speed, torque limit
  // heightfield
  int hf_nrow, hf_ncol;
  float hf_hx, hf_hy;
  const float *hf_data;                // [nrow][ncol]
  const int *hf_convex;                // [nrow][ncol] 1: convex interior vertex (box-face contacts)
  // body tree
  const int *body_parent, *body_jnt, *body_root, *body_dl, *level_body, *level_start;
  // [nbody - 1][4] per entry of level_body: body | parent << 16, joint (-1: none),
  // joint type (255: none) | qpos address << 8, dof address | child_start << 12 | children << 24
  const int *level_rec;
  const int *child_start, *child_list;
  const int *body_geom_adr, *body_geom;  // [nbody + 1], [ngeom] geoms of each body
  const float *body_pos, *body_quat, *body_mass, *body_ipos, *body_inertia;
  // joints and dofs
  const int *jnt_type, *jnt_qadr, *jnt_dadr;
  const float *jnt_axis, *jnt_pos, *jnt_noise, *qpos_reset;
  const int *dof_body, *dof_jnt, *dof_rowadr, *dof_rowlen, *colind, *entry_row;
  const int *col_start, *col_k, *col_pos;
  const float *dof_armature;
  // actuators
  const int *act_qadr, *act_dadr;
  const float *act_kp, *act_kd;
  // geoms and pairs
  const int *geom_type, *geom_body;
  const float *geom_size, *geom_pos, *geom_mat, *geom_friction;
  const int *pair_g1, *pair_g2;
  // packed update lists: LTDL elimination of dof k (pairs 1 <= p <= q < len_k) and the
  // chain outer product of a contact on the chain ending at dof d (pairs 0 <= p <= q < len_d);
  // each op = target entry | p << 12 | q << 17
  const int *ltdl_adr, *chain_adr;
  const unsigned *ltdl_ops, *chain_ops;
  const unsigned long long *body_mask;   // bit d set when dof d moves body b
  const unsigned long long *dof_mask;    // bit i set when dof i is dof d or one of its ancestors
  const int *tri_pq;                      // t -> p | q << 5 for 0 <= p <= q < 32, t = q (q + 1) / 2 + p
  // full symmetric rows of M: row i's ops sym_ops[sym_start[i] .. sym_start[i + 1]), each
  // stored entry | column dof << 12 -- the row's own entries, then its descendants' column-i
  // entries (the order of the sums of M x)
  const int *sym_start;
  const unsigned *sym_ops;
  const unsigned *entry_ops;   // [nM] row's diagonal entry | row << 12 | column << 18
};

// Per-world contact record in shared memory (floats); odd stride avoids bank conflicts
enum {
  C_POS = 0, C_FRAME = 3, C_DIST = 12, C_MU = 13, C_D = 14, C_AREF = 15, C_JAR = 18,
  C_JV = 21, C_F = 24, C_HC = 27, C_FS = 33, C_STRIDE = 39
};
// Per-world contact integer record (MLO/MHI, M1LO/M1HI: chain bit masks of bodies 2, 1)
enum { CI_G1 = 0, CI_G2 = 1, CI_B1 = 2, CI_B2 = 3, CI_MLO = 4, CI_MHI = 5, CI_M1LO = 6, CI_M1HI = 7, CI_STRIDE = 8 };
// Per-world joint-limit row (floats; the dof is stored as int bits)
enum { LM_DOF = 0, LM_SIGN, LM_DIST, LM_D, LM_AREF, LM_JAR, LM_JV, LM_F, LM_STRIDE = 8 };
// per-body dynamics record: cinert, then {cacc, cfrc} during RNE, reused by crb for CRBA
// (U_REL: the joints' relative transforms, 7 floats, during forward kinematics)
enum { U_CINERT = 0, U_CACC = 10, U_CFRC = 16, U_CRB = 10, U_REL = 10, U_STRIDE = 23 };
// the grouped smooth launches' shared block (per world): AUX_CI floats per body of com (then
// composite) inertia, then a region of aux_region_floats() reused over time; odd strides keep
// the lanes' per-body and per-dof accesses on distinct banks
enum { AUX_CI = 11, AUX_R = 7 };
static inline B3P_HD int aux_region_floats(int nb, int nv) {
  return 2 * AUX_R * nb > AUX_R * nv ? 2 * AUX_R * nb : AUX_R * nv;
}
#define B3P_OPS_TARGET(op) ((int)((op) & 0xfffu))
#define B3P_OPS_P(op) ((int)(((op) >> 12) & 31u))
#define B3P_OPS_Q(op) ((int)(((op) >> 17) & 31u))
// FP64 pivot-fallback workspace per world (doubles): H (tree rows or dense) and one vector
#define B3P_SCRATCH_DOUBLES(nM, nv, dense) ((dense) ? (nv) * (nv) + (nv) : (nM) + (nv))

// Lane-per-world Newton solve: one world per lane, 32 worlds per warp, each world's solve
// data in shared memory as [element][33] floats (element e of lane l at 33 e + l: bank
// (e + l) mod 32, conflict-free both for one element of all lanes and for consecutive
// elements of one lane). Elements: M's factor, H's factor, M's diagonal, seven dof vectors,
// one chain's H_c J products, and B3P_LANE_NCL contact records with their Jacobian rows.
#define B3P_LANE_NCL 8
#define B3P_LANE_STRIDE 33
enum { LK_MU = 0, LK_D = 1, LK_AREF = 2, LK_JAR = 5, LK_JV = 8, LK_HC = 11, LK_F = 17, LK_B2 = 20, LK_J = 21 };
struct LaneLayout {
  int L, F, Md, a, qs, frc, Ma, Mp, g, p, w, con, cstride, total;
};
B3P_HD inline LaneLayout lane_layout(int nM, int nv, int maxchain) {
  LaneLayout o;
  int off = 0;
  o.L = off; off += nM;
  o.F = off; off += nM;
  o.Md = off; off += nv;
  o.a = off; off += nv;
  o.qs = off; off += nv;
  o.frc = off; off += nv;
  o.Ma = off; off += nv;
  o.Mp = off; off += nv;
  o.g = off; off += nv;
  o.p = off; off += nv;
  o.w = off; off += 3 * maxchain;
  o.cstride = LK_J + 3 * maxchain;
  o.con = off; off += B3P_LANE_NCL * o.cstride;
  o.total = off;
  return o;
}

// One model group of a batch: world range and its per-world arrays.
struct DGroup {
  const DModel *m;
  int world_start, nworld, ctrl_offset;
  int ws_off4;         // offset of the group's global working sets, in units of 4 floats
  float *qpos, *qvel, *qacc;
  int *step_count, *rng_id;
  uint32_t *seed;      // [W][2]
  uint32_t *status;
  int *stats;          // [W][4]
  float *friction, *mass_scale, *kp, *kd;
  float *inertia;      // [W][nb][10] mass, com (3), inertia (6) per body
  int inertia_custom;  // 0: every world's entries are the model's own (never set), so the
                       // kernels read the model's constants instead of W copies of them
  float *con;          // [W][ncon_max][24] or null
  int *ncon;           // [W] or null
  double *scratch64;   // [W][nM + nv] FP64 pivot-fallback workspace
  float *ctrl_hist;    // [W][act_delay][nu_pad] delayed targets (null without delay)
  float *state_hist;   // [W][history][nq + nv] ring of recent states (null without history)
  int history;
  int lane_ok;         // the group's solves may run one world per lane (tree Hessian, no limits)
};

struct DBatch {
  int ngroup, nworld, smem_floats, schedule;  // schedule 1: dynamic queue over `order`
  int *counter;                               // next queue position (zeroed before each launch)
  const int *order;                           // [nworld] world indices, heaviest models first
  float *ws;                                  // working sets in global memory (null: shared memory)
  long long ws_floats;
  int *solve_order;                           // staged, schedule 1: worlds by contact count, most first
  unsigned char *solve_key;                   // [nworld] bucket of each world (collide launch)
  int aux_floats;                             // per-world launch-local scratch: max over groups
                                              // of pad4(AUX_CI nb + aux_region_floats(nb, nv))
  int solve_aux_floats;                       // per-world Newton arrays: max over groups of
                                              // pad4(nv nv dense | nM tree) + 5 pad4(nv), and
                                              // with staged inputs 2 pad4(nM) + pad4(6 nv)
  int lane_solve;                             // 1: worlds with 1..B3P_LANE_NCL rows of lane_ok
                                              // groups are solved one per lane
  int *lane_order;                            // [nworld + 32 ngroup] those worlds, per group in
                                              // segments padded to whole warps (-1: padding)
  int *solve_counts;                          // [2] worlds in solve_order, entries of lane_order
  DGroup g[B3P_MAXGROUP];
};

// kernel-side entry points (b3p_step.cu); return a cudaError_t value
extern "C" int b3p_launch_step(const DBatch *dbatch_dev, int nworld, const float *ctrl, int decimation,
                               int warps_per_block, int grid, int smem_bytes, void *stream);
extern "C" int b3p_launch_reset(const DBatch *dbatch_dev, int nworld, uint32_t seed_lo, uint32_t seed_hi,
                                const int *world_ids, const int *rng_ids, int n, void *stream);
extern "C" int b3p_step_occupancy(int smem_bytes, int warps_per_block, int *blocks_per_sm);
// per-group offsets (floats) of the global working-set region: world wi of group g uses
// ws + ws_offset[g] + lw * smem_floats_g
// lim: a model of the launch has limited joints (selects the solve kernel that handles them)
extern "C" int b3p_launch_plain(const DBatch *b, int group, int nworld, const float *ctrl, int decimation, float *ws,
                                int lim, void *stream);
// sorted: the solve stage takes worlds by constraint-row count, most first (schedule 1)
// grouped: consecutive per-world stages share a launch (working_set 3)
// lane_smem > 0: the solve runs one world per lane where it can (lane_solve batches), with
// that many bytes of dynamic shared memory per 32-world CTA
// aux_smem > 0 (grouped staging): the smooth-dynamics launches keep each world's launch-local
// scratch (composite inertias and RNE terms, the CRBA temporary, body quaternions) in that
// many bytes of dynamic shared memory per CTA instead of the working set
// solve_smem > 0: the solve launch keeps each world's launch-local Newton arrays (H or its
// factor, pivot thresholds, M a, M p, gradient, direction) in that many bytes per CTA
// one_model: the batch holds one model group (its limit-free solve launch then uses the
// instantiation compiled for 7 resident CTAs)
extern "C" int b3p_launch_staged(const DBatch *b, int nworld, const float *ctrl, int decimation, int wpb,
                                 int lim, int sorted, int grouped, int lane_smem, int aux_smem, int solve_smem,
                                 int one_model, void *stream);
extern "C" int b3p_aux_prepare(int bytes);
extern "C" int b3p_solve_aux_prepare(int bytes);
extern "C" int b3p_aux_fits(int smooth_bytes, int solve_bytes, int wpb, int *smooth_ok, int *solve_ok);
// the same launches with events[k] recorded before launch k and events[2 + 6 d] after
// the last (events: 3 + 6 d created events)
extern "C" int b3p_launch_staged_events(const DBatch *b, int nworld, const float *ctrl, int decimation, int wpb,
                                        int lim, int sorted, int lane_smem, int solve_smem, int one_model,
                                        void *stream, void *const *events);
// lift the lane solve kernel's dynamic shared-memory limit to `bytes` (once per batch)
extern "C" int b3p_lane_solve_prepare(int bytes);
extern "C" int b3p_launch_observe(const DBatch *b, int group, int nworld, int width, const float *ctrl, float *out,
                                  void *stream);
extern "C" int b3p_launch_sensor(const DBatch *b, int group, int nworld, const int *bodies, int n, float threshold,
                                 float dt, float *state, float *force, float *hist, int depth, void *stream);
// reward and termination (b3p_reward): the configuration and buffers, passed by value
#define B3P_NTERMS 10
#define B3P_NBODYLIST 16
struct RewardArgs {
  float weight[B3P_NTERMS];
  float sigma_lin, sigma_ang, air_time_target, dt, min_height, max_tilt;
  int max_steps, nfeet, nillegal;
  int feet[B3P_NBODYLIST], illegal[B3P_NBODYLIST];
  const float *cmd, *action, *prev, *sensor;
  float *reward, *terms, *episode;
  uint32_t *done;
};
extern "C" int b3p_launch_reward(const DBatch *b, int group, int nworld, int smem_floats, const RewardArgs *args,
                                 void *stream);
extern "C" int b3p_launch_diffik(const DBatch *b, int group, int nworld, int smem_floats, int body, float ox, float oy,
                                 float oz, const float *tpos, const float *tquat, float lambda, float *ctrl,
                                 void *stream);
// flags: 1 world geoms only, 2 no bounding-volume hierarchy; hitpos / hitnrm may be null
extern "C" int b3p_launch_raycast(const DBatch *b, int group, int nworld, int smem_floats, int body, int nray,
                                  const float *org, const float *dir, float max_dist, int flags, float *dist,
                                  float *hitpos, float *hitnrm, void *stream);
extern "C" int b3p_launch_history(const DBatch *b, int group, int world, float *dst, int *count, void *stream);
extern "C" int b3p_launch_idle(const DBatch *b, const int *ids, int n, int idle, void *stream);
extern "C" int b3p_launch_targets(const DBatch *b, int nworld, const float *sigma_dev, float *ctrl, void *stream);
extern "C" int b3p_launch_gather(const DBatch *b, int group, int field, const int *ids, int n, int width,
                                 float *dst, void *stream);
// grid: the static kernel's own occupancy (blocks per SM for warps_per_block and
// smem_bytes) times the SM count, capped by the CTAs the worlds fill
extern "C" int b3p_launch_step_static(const DBatch *dbatch_dev, int nworld, const float *ctrl, int decimation,
                                      int warps_per_block, int smem_bytes, void *stream);
// FP32 FMA throughput of the current device (b3p_fp32_peak)
extern "C" int b3p_fma_probe(int reps, double *flops_per_s, int *sm_count, void *stream);
