// FP64 CPU oracle for the batched rigid-body step -- TEST INFRASTRUCTURE ONLY.
//
// Used by tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg; the
// product path never links or loads it, and it shares no code with the CUDA
// library. Plain, slow and direct: dense matrices, definitions written out,
// no blocking or fusion. Each function names what it follows.
//
// Reference frame: every spatial vector is expressed in world orientation about
// the world origin O. Motion vectors are [angular; linear], force vectors
// [moment; force] (Featherstone, "Rigid Body Dynamics Algorithms", 2008, ch. 2).
// The physics step order follows MuJoCo's documented pipeline (kinematics,
// inertia, bias, actuation, collision, constraint solve, semi-implicit Euler);
// the mjlab paper (arXiv 2601.22074, Architecture) only states that N
// independent worlds share one model and advance together.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

namespace {

enum { FREE = 0, HINGE = 1, SLIDE = 2 };
enum { PLANE = 0, SPHERE = 1, CAPSULE = 2, BOX = 3, HFIELD = 4 };
enum { ST_NAN = 1, ST_OVERFLOW = 2, ST_NOCONV = 4 };
enum { PURPOSE_RESET = 1, PURPOSE_PUSH = 2 };

struct Model {
  int nb = 0, nj = 0, nu = 0, ng = 0, nq = 0, nv = 0;
  std::vector<int> parent, body_jnt, jtype, jbody, qadr, dadr, act_jnt, gtype, gbody;
  std::vector<double> bpos, bquat, bmass, bipos, binertia;
  std::vector<double> jaxis, jpos, jarm, jnoise, qpos_reset, kp, kd;
  std::vector<double> gsize, gpos, gquat, gfric;
  std::vector<uint32_t> ct, ca;
  std::vector<int> dof_body, dof_jnt, dof_parent;
  std::vector<int> pairs;  // [npair][2]
  int ncon_max = 0;
  double h = 0, grav[3] = {0, 0, 0}, solref[2] = {0, 0}, solimp[5] = {0, 0, 0, 0, 0};
  int newton_iter = 0, ls_iter = 0, cap = 0, push_period = 0;
  double newton_tol = 0, pivot_tau = 0, push_sigma = 0;
  std::vector<int> jlimited;   // [nj]
  std::vector<double> jrange;  // [nj][2]
  std::vector<double> dcm;     // [nu][3] stall torque, no-load speed, torque limit
  int hf_nrow = 0, hf_ncol = 0;
  double hf_size[2] = {0, 0};
  std::vector<double> hf;      // [nrow][ncol]
  std::vector<char> hf_convex; // [nrow][ncol] 1: interior vertex above the mean of its 4 neighbours
};

// ------------------------------------------------------------------ small vector math
inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross3(const double *a, const double *b, double *o) {
  double r[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  o[0] = r[0]; o[1] = r[1]; o[2] = r[2];
}
inline void matvec3(const double *R, const double *v, double *o) {  // row-major R
  double r[3];
  for (int i = 0; i < 3; i++) r[i] = R[3 * i] * v[0] + R[3 * i + 1] * v[1] + R[3 * i + 2] * v[2];
  o[0] = r[0]; o[1] = r[1]; o[2] = r[2];
}
inline void matmul3(const double *A, const double *B, double *C) {
  double r[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) r[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
  std::memcpy(C, r, sizeof r);
}
inline void quat_mul(const double *a, const double *b, double *o) {  // Hamilton, (w,x,y,z)
  double r[4] = {a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                 a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                 a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                 a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]};
  std::memcpy(o, r, sizeof r);
}
inline void quat_normalize(double *q) {
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (n > 0) for (int i = 0; i < 4; i++) q[i] /= n;
}
inline void quat2mat(const double *q, double *R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
inline void axis_angle_quat(const double *axis, double ang, double *q) {
  double n = std::sqrt(dot3(axis, axis));
  double s = std::sin(0.5 * ang) / n;
  q[0] = std::cos(0.5 * ang); q[1] = axis[0] * s; q[2] = axis[1] * s; q[3] = axis[2] * s;
}
// spatial cross products (Featherstone 2.9): motion x motion, motion x* force
inline void crossm(const double *v, const double *m, double *o) {
  double a[3], b[3], c[3];
  cross3(v, m, a);
  cross3(v, m + 3, b);
  cross3(v + 3, m, c);
  o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
  o[3] = b[0] + c[0]; o[4] = b[1] + c[1]; o[5] = b[2] + c[2];
}
inline void crossf(const double *v, const double *f, double *o) {
  double a[3], b[3], c[3];
  cross3(v, f, a);
  cross3(v + 3, f + 3, b);
  cross3(v, f + 3, c);
  o[0] = a[0] + b[0]; o[1] = a[1] + b[1]; o[2] = a[2] + b[2];
  o[3] = c[0]; o[4] = c[1]; o[5] = c[2];
}
inline void mat6vec(const double *A, const double *v, double *o) {
  for (int i = 0; i < 6; i++) {
    double s = 0;
    for (int j = 0; j < 6; j++) s += A[6 * i + j] * v[j];
    o[i] = s;
  }
}

// ------------------------------------------------------------------ Philox-4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11:
// ten rounds of the 4x32 S-box with multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key
// increments 0x9E3779B9, 0xBB67AE85.
void philox(const uint32_t c_in[4], const uint32_t k_in[2], uint32_t out[4]) {
  uint32_t c[4] = {c_in[0], c_in[1], c_in[2], c_in[3]};
  uint32_t k[2] = {k_in[0], k_in[1]};
  for (int r = 0; r < 10; r++) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n[4] = {hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0};
    std::memcpy(c, n, sizeof n);
  }
  std::memcpy(out, c, sizeof c);
}
inline double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// ------------------------------------------------------------------ per-world kinematics
struct Kin {
  std::vector<double> xpos, xquat, xmat, xipos, gxpos, gxmat, cdof, I6;
  void init(const Model &m) {
    xpos.assign(3 * m.nb, 0); xquat.assign(4 * m.nb, 0); xmat.assign(9 * m.nb, 0);
    xipos.assign(3 * m.nb, 0); gxpos.assign(3 * m.ng, 0); gxmat.assign(9 * m.ng, 0);
    cdof.assign(6 * m.nv, 0); I6.assign(36 * m.nb, 0);
  }
};

bool is_ancestor_or_self(const Model &m, int anc, int b) {
  while (b >= 0) {
    if (b == anc) return true;
    b = m.parent[b];
  }
  return false;
}

// Forward kinematics (MuJoCo's joint conventions): free joint qpos = world position
// and orientation; a hinge rotates the body about its axis through the anchor, keeping
// the anchor fixed; a slide translates along its axis.
void kinematics(const Model &m, const double *qpos, Kin &k) {
  k.xpos[0] = k.xpos[1] = k.xpos[2] = 0;
  k.xquat[0] = 1; k.xquat[1] = k.xquat[2] = k.xquat[3] = 0;
  quat2mat(&k.xquat[0], &k.xmat[0]);
  for (int b = 1; b < m.nb; b++) {
    int j = m.body_jnt[b], p = m.parent[b];
    double pos[3], quat[4];
    if (j >= 0 && m.jtype[j] == FREE) {
      const double *q = qpos + m.qadr[j];
      pos[0] = q[0]; pos[1] = q[1]; pos[2] = q[2];
      quat[0] = q[3]; quat[1] = q[4]; quat[2] = q[5]; quat[3] = q[6];
      quat_normalize(quat);
    } else {
      matvec3(&k.xmat[9 * p], &m.bpos[3 * b], pos);
      for (int i = 0; i < 3; i++) pos[i] += k.xpos[3 * p + i];
      quat_mul(&k.xquat[4 * p], &m.bquat[4 * b], quat);
      quat_normalize(quat);
      if (j >= 0 && m.jtype[j] == HINGE) {
        double R[9], anchor[3], qa[4], q2[4], R2[9], off[3];
        quat2mat(quat, R);
        matvec3(R, &m.jpos[3 * j], anchor);
        for (int i = 0; i < 3; i++) anchor[i] += pos[i];
        axis_angle_quat(&m.jaxis[3 * j], qpos[m.qadr[j]], qa);
        quat_mul(quat, qa, q2);
        quat_normalize(q2);
        quat2mat(q2, R2);
        matvec3(R2, &m.jpos[3 * j], off);
        for (int i = 0; i < 3; i++) pos[i] = anchor[i] - off[i];
        std::memcpy(quat, q2, sizeof q2);
      } else if (j >= 0 && m.jtype[j] == SLIDE) {
        double R[9], ax[3];
        quat2mat(quat, R);
        matvec3(R, &m.jaxis[3 * j], ax);
        double n = std::sqrt(dot3(ax, ax));
        for (int i = 0; i < 3; i++) pos[i] += ax[i] / n * qpos[m.qadr[j]];
      }
    }
    std::memcpy(&k.xpos[3 * b], pos, sizeof pos);
    std::memcpy(&k.xquat[4 * b], quat, sizeof quat);
    quat2mat(quat, &k.xmat[9 * b]);
    double ip[3];
    matvec3(&k.xmat[9 * b], &m.bipos[3 * b], ip);
    for (int i = 0; i < 3; i++) k.xipos[3 * b + i] = pos[i] + ip[i];
  }
  for (int g = 0; g < m.ng; g++) {
    int b = m.gbody[g];
    double off[3], Rg[9];
    matvec3(&k.xmat[9 * b], &m.gpos[3 * g], off);
    for (int i = 0; i < 3; i++) k.gxpos[3 * g + i] = k.xpos[3 * b + i] + off[i];
    quat2mat(&m.gquat[4 * g], Rg);
    matmul3(&k.xmat[9 * b], Rg, &k.gxmat[9 * g]);
  }
}

// Motion subspace of every dof as a spatial motion vector about O (world orientation).
// Hinge: [a; p x a] with a the world axis, p the anchor; slide: [0; a]; free joint:
// translation along the world axes, rotation about the body axes (qvel of a free
// joint holds the world linear velocity of the body origin and the body-frame
// angular velocity, MuJoCo's convention).
void motion_subspace(const Model &m, Kin &k) {
  for (int j = 0; j < m.nj; j++) {
    int b = m.jbody[j], d = m.dadr[j];
    const double *R = &k.xmat[9 * b];
    const double *xp = &k.xpos[3 * b];
    if (m.jtype[j] == FREE) {
      for (int i = 0; i < 3; i++) {
        double *s = &k.cdof[6 * (d + i)];
        std::fill(s, s + 6, 0.0);
        s[3 + i] = 1;
      }
      for (int i = 0; i < 3; i++) {
        double a[3] = {R[i], R[3 + i], R[6 + i]};
        double *s = &k.cdof[6 * (d + 3 + i)];
        s[0] = a[0]; s[1] = a[1]; s[2] = a[2];
        cross3(xp, a, s + 3);
      }
    } else {
      double a[3];
      matvec3(R, &m.jaxis[3 * j], a);
      double n = std::sqrt(dot3(a, a));
      for (int i = 0; i < 3; i++) a[i] /= n;
      double *s = &k.cdof[6 * d];
      if (m.jtype[j] == HINGE) {
        double anc[3];
        matvec3(R, &m.jpos[3 * j], anc);
        for (int i = 0; i < 3; i++) anc[i] += xp[i];
        s[0] = a[0]; s[1] = a[1]; s[2] = a[2];
        cross3(anc, a, s + 3);
      } else {
        s[0] = s[1] = s[2] = 0;
        s[3] = a[0]; s[4] = a[1]; s[5] = a[2];
      }
    }
  }
}

// Spatial inertia of each body about O: [[Ic + m(c.c 1 - c c^T), m[c]x], [m[c]x^T, m 1]]
// with c the world centre of mass and Ic = R I_body R^T (RBDA eq. 2.63).
void spatial_inertia(const Model &m, const double *mass_scale, Kin &k) {
  for (int b = 0; b < m.nb; b++) {
    double *A = &k.I6[36 * b];
    std::fill(A, A + 36, 0.0);
    double s = mass_scale ? mass_scale[b] : 1.0;
    double mass = m.bmass[b] * s;
    if (b == 0 || mass <= 0) continue;
    const double *in = &m.binertia[6 * b];
    double Ib[9] = {in[0], in[3], in[4], in[3], in[1], in[5], in[4], in[5], in[2]};
    for (int i = 0; i < 9; i++) Ib[i] *= s;
    const double *R = &k.xmat[9 * b];
    double Rt[9] = {R[0], R[3], R[6], R[1], R[4], R[7], R[2], R[5], R[8]};
    double T[9], Ic[9];
    matmul3(R, Ib, T);
    matmul3(T, Rt, Ic);
    const double *c = &k.xipos[3 * b];
    double cc = dot3(c, c);
    double cx[9] = {0, -c[2], c[1], c[2], 0, -c[0], -c[1], c[0], 0};
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        A[6 * i + j] = Ic[3 * i + j] + mass * ((i == j ? cc : 0) - c[i] * c[j]);
        A[6 * i + 3 + j] = mass * cx[3 * i + j];
        A[6 * (3 + i) + j] = mass * cx[3 * j + i];
        A[6 * (3 + i) + 3 + j] = (i == j) ? mass : 0;
      }
  }
}

// body Jacobian column: dof d moves body b iff the dof's body is b or an ancestor.
inline bool dof_moves(const Model &m, int d, int b) { return is_ancestor_or_self(m, m.dof_body[d], b); }

// M = sum_b J_b^T I_b J_b + diag(armature)
void mass_matrix(const Model &m, const Kin &k, double *M) {
  int nv = m.nv;
  std::fill(M, M + nv * nv, 0.0);
  std::vector<double> IJ(6 * nv);
  for (int b = 1; b < m.nb; b++) {
    for (int d = 0; d < nv; d++) {
      double *o = &IJ[6 * d];
      if (dof_moves(m, d, b)) mat6vec(&k.I6[36 * b], &k.cdof[6 * d], o);
      else std::fill(o, o + 6, 0.0);
    }
    for (int r = 0; r < nv; r++) {
      if (!dof_moves(m, r, b)) continue;
      for (int c = 0; c < nv; c++) {
        double s = 0;
        for (int i = 0; i < 6; i++) s += k.cdof[6 * r + i] * IJ[6 * c + i];
        M[r * nv + c] += s;
      }
    }
  }
  for (int d = 0; d < nv; d++) M[d * nv + d] += m.jarm[m.dof_jnt[d]];
}

// body spatial velocity v_b = J_b qvel
void body_velocity(const Model &m, const Kin &k, int b, const double *qvel, double *v) {
  std::fill(v, v + 6, 0.0);
  for (int d = 0; d < m.nv; d++)
    if (dof_moves(m, d, b))
      for (int i = 0; i < 6; i++) v[i] += k.cdof[6 * d + i] * qvel[d];
}

// Inverse dynamics tau = sum_b J_b^T (I_b a_b + v_b x* I_b v_b), with
// a_b = J_b qacc + sum_d sdot_d qvel_d + a_grav; sdot_d = v_ref x s_d where v_ref is the
// velocity of the body in which the axis is fixed (the parent for hinge/slide, the
// body itself for free-joint rotations, none for free-joint translations).
void inverse_dynamics(const Model &m, const Kin &k, const double *qvel, const double *qacc,
                      bool gravity, double *tau) {
  int nv = m.nv;
  std::vector<double> vb(6 * m.nb, 0.0), sdot(6 * nv, 0.0);
  for (int b = 1; b < m.nb; b++) body_velocity(m, k, b, qvel, &vb[6 * b]);
  for (int d = 0; d < nv; d++) {
    int j = m.dof_jnt[d], b = m.dof_body[d];
    double *o = &sdot[6 * d];
    if (m.jtype[j] == FREE) {
      if (d - m.dadr[j] < 3) continue;
      crossm(&vb[6 * b], &k.cdof[6 * d], o);
    } else {
      crossm(&vb[6 * m.parent[b]], &k.cdof[6 * d], o);
    }
  }
  std::fill(tau, tau + nv, 0.0);
  for (int b = 1; b < m.nb; b++) {
    double a[6] = {0, 0, 0, 0, 0, 0};
    if (gravity) for (int i = 0; i < 3; i++) a[3 + i] = -m.grav[i];
    for (int d = 0; d < nv; d++)
      if (dof_moves(m, d, b))
        for (int i = 0; i < 6; i++) a[i] += k.cdof[6 * d + i] * qacc[d] + sdot[6 * d + i] * qvel[d];
    double f[6], Iv[6], vxIv[6];
    mat6vec(&k.I6[36 * b], a, f);
    mat6vec(&k.I6[36 * b], &vb[6 * b], Iv);
    crossf(&vb[6 * b], Iv, vxIv);
    for (int i = 0; i < 6; i++) f[i] += vxIv[i];
    for (int d = 0; d < nv; d++)
      if (dof_moves(m, d, b)) {
        double s = 0;
        for (int i = 0; i < 6; i++) s += k.cdof[6 * d + i] * f[i];
        tau[d] += s;
      }
  }
}

// dense LDL^T (no pivoting) of an SPD matrix; returns false on a non-positive pivot
bool dense_ldl(int n, const double *A, std::vector<double> &L, std::vector<double> &D) {
  L.assign(n * n, 0.0);
  D.assign(n, 0.0);
  for (int j = 0; j < n; j++) {
    double s = A[j * n + j];
    for (int k = 0; k < j; k++) s -= L[j * n + k] * L[j * n + k] * D[k];
    if (!(s > 0)) return false;
    D[j] = s;
    L[j * n + j] = 1;
    for (int i = j + 1; i < n; i++) {
      double t = A[i * n + j];
      for (int k = 0; k < j; k++) t -= L[i * n + k] * L[j * n + k] * D[k];
      L[i * n + j] = t / s;
    }
  }
  return true;
}
void dense_ldl_solve(int n, const std::vector<double> &L, const std::vector<double> &D, double *x) {
  for (int i = 0; i < n; i++)
    for (int k = 0; k < i; k++) x[i] -= L[i * n + k] * x[k];
  for (int i = 0; i < n; i++) x[i] /= D[i];
  for (int i = n - 1; i >= 0; i--)
    for (int k = i + 1; k < n; k++) x[i] -= L[k * n + i] * x[k];
}

// ------------------------------------------------------------------ collision
struct Contact {
  int g1, g2, b1, b2;
  double dist, pos[3], frame[9], mu;
  double force[3];
};

// tangent frame: t1 = normalise(n x e_k), e_k the world axis least aligned with n
// (lowest index on ties), t2 = n x t1.
void contact_frame(const double *n, double *frame) {
  int k = 0;
  double best = std::fabs(n[0]);
  for (int i = 1; i < 3; i++)
    if (std::fabs(n[i]) < best) { best = std::fabs(n[i]); k = i; }
  double e[3] = {0, 0, 0};
  e[k] = 1;
  double t1[3], t2[3];
  cross3(n, e, t1);
  double l = std::sqrt(dot3(t1, t1));
  for (int i = 0; i < 3; i++) t1[i] /= l;
  cross3(n, t1, t2);
  for (int i = 0; i < 3; i++) { frame[i] = n[i]; frame[3 + i] = t1[i]; frame[6 + i] = t2[i]; }
}

void plane_point(const double *n, const double *p0, const double *c, double r,
                 std::vector<Contact> &out, Contact proto) {
  double diff[3] = {c[0] - p0[0], c[1] - p0[1], c[2] - p0[2]};
  double dist = dot3(n, diff) - r;
  if (dist < 0) {
    proto.dist = dist;
    for (int i = 0; i < 3; i++) proto.pos[i] = c[i] - n[i] * (r + 0.5 * dist);
    contact_frame(n, proto.frame);
    out.push_back(proto);
  }
}

// Box-box narrow phase (separating-axis test, then a contact manifold).
// Axes: 0-2 face normals of box A (geom1), 3-5 of box B, 6-14 the normalised cross
// products a_i x b_j (index 6 + 3 i + j; skipped when |a_i x b_j| < 1e-6). Overlap
// along a unit axis L: sum_k hA_k |a_k.L| + sum_k hB_k |b_k.L| - |(cB - cA).L|; any
// negative overlap separates the boxes. Chosen axis (reading of "minimum penetration,
// ties to the lowest index", with a preference that keeps the choice stable between
// precisions): the best face of A unless B's best face is smaller by more than 0.1 %,
// then an edge axis only when its overlap is more than 5 % smaller than that face's.
// Face case: the reference face is the chosen face (normal pointing to the other box);
// the incident face is the other box's face most anti-parallel to it (lowest index on
// ties); the incident quad (vertex order (-,-) (+,-) (+,+) (-,+)) is clipped against the
// reference face's side planes (+u, -u, +v, -v; Sutherland-Hodgman) and every clipped
// point below the reference face is a contact at the midpoint to its projection.
// Edge case: one contact at the midpoint of the closest points of the two supporting
// edges (segment parameters clamped to the edge lengths). The normal points from A to B.
// Returns the contact count; axis_out / minov_out report the chosen axis and the
// smallest overlap over all valid axes (for tests).
int box_box(const double *cA, const double *RA, const double *hA, const double *cB, const double *RB,
            const double *hB, std::vector<Contact> &out, Contact proto, int *axis_out, double *minov_out) {
  double a[3][3], b[3][3], d[3];
  for (int i = 0; i < 3; i++)
    for (int r = 0; r < 3; r++) { a[i][r] = RA[3 * r + i]; b[i][r] = RB[3 * r + i]; }
  for (int r = 0; r < 3; r++) d[r] = cB[r] - cA[r];
  double L[15][3], ov[15];
  bool valid[15];
  double minov = 1e300;
  for (int k = 0; k < 15; k++) {
    valid[k] = true;
    if (k < 3) { for (int r = 0; r < 3; r++) L[k][r] = a[k][r]; }
    else if (k < 6) { for (int r = 0; r < 3; r++) L[k][r] = b[k - 3][r]; }
    else {
      cross3(a[(k - 6) / 3], b[(k - 6) % 3], L[k]);
      double n = std::sqrt(dot3(L[k], L[k]));
      if (n < 1e-6) { valid[k] = false; continue; }
      for (int r = 0; r < 3; r++) L[k][r] /= n;
    }
    double rA = 0, rB = 0;
    for (int q = 0; q < 3; q++) { rA += hA[q] * std::fabs(dot3(a[q], L[k])); rB += hB[q] * std::fabs(dot3(b[q], L[k])); }
    ov[k] = rA + rB - std::fabs(dot3(d, L[k]));
    if (ov[k] < 0) { if (axis_out) *axis_out = -1; if (minov_out) *minov_out = ov[k]; return 0; }
    minov = std::min(minov, ov[k]);
  }
  if (minov_out) *minov_out = minov;
  int fa = 0, fb = 3, e = -1;
  for (int k = 1; k < 3; k++) if (ov[k] < ov[fa]) fa = k;
  for (int k = 4; k < 6; k++) if (ov[k] < ov[fb]) fb = k;
  for (int k = 6; k < 15; k++) if (valid[k] && (e < 0 || ov[k] < ov[e])) e = k;
  int best = (ov[fb] * 1.001 < ov[fa]) ? fb : fa;
  if (e >= 0 && ov[e] * 1.05 < ov[best]) best = e;
  if (axis_out) *axis_out = best;
  int n0 = (int)out.size();
  if (best < 6) {
    bool refA = best < 3;
    const double(*R)[3] = refA ? a : b;    // reference box axes
    const double(*I)[3] = refA ? b : a;    // incident box axes
    const double *cR0 = refA ? cA : cB, *cI0 = refA ? cB : cA, *hR = refA ? hA : hB, *hI = refA ? hB : hA;
    int i = refA ? best : best - 3;
    double toward[3] = {cI0[0] - cR0[0], cI0[1] - cR0[1], cI0[2] - cR0[2]};
    double sg = dot3(toward, R[i]) >= 0 ? 1.0 : -1.0;
    double nr[3] = {sg * R[i][0], sg * R[i][1], sg * R[i][2]};
    double cR[3] = {cR0[0] + hR[i] * nr[0], cR0[1] + hR[i] * nr[1], cR0[2] + hR[i] * nr[2]};
    int ui = (i + 1) % 3, vi = (i + 2) % 3;
    int kI = 0;
    double best_abs = -1;
    for (int k = 0; k < 3; k++) {
      double dk = std::fabs(dot3(I[k], nr));
      if (dk > best_abs) { best_abs = dk; kI = k; }
    }
    double so = dot3(I[kI], nr) >= 0 ? -1.0 : 1.0;   // outward normal so * I[kI] faces the reference
    int e1 = (kI + 1) % 3, e2 = (kI + 2) % 3;
    double cI[3];
    for (int r = 0; r < 3; r++) cI[r] = cI0[r] + so * hI[kI] * I[kI][r];
    double poly[8][3];
    int np = 4;
    const double sgn[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    for (int q = 0; q < 4; q++)
      for (int r = 0; r < 3; r++) poly[q][r] = cI[r] + sgn[q][0] * hI[e1] * I[e1][r] + sgn[q][1] * hI[e2] * I[e2][r];
    const int plane_axis[4] = {ui, ui, vi, vi};
    const double plane_sign[4] = {1, -1, 1, -1};
    for (int pl = 0; pl < 4 && np > 0; pl++) {
      const double *ax = R[plane_axis[pl]];
      double half = hR[plane_axis[pl]], ps = plane_sign[pl];
      double outp[8][3];
      int no = 0;
      for (int q = 0; q < np; q++) {
        const double *P = poly[q], *Q = poly[(q + 1) % np];
        double dP[3] = {P[0] - cR[0], P[1] - cR[1], P[2] - cR[2]}, dQ[3] = {Q[0] - cR[0], Q[1] - cR[1], Q[2] - cR[2]};
        double fP = ps * dot3(dP, ax) - half, fQ = ps * dot3(dQ, ax) - half;
        if (fP <= 0 && no < 8) { for (int r = 0; r < 3; r++) outp[no][r] = P[r]; no++; }
        if (((fP < 0 && fQ > 0) || (fP > 0 && fQ < 0)) && no < 8) {
          double t = fP / (fP - fQ);
          for (int r = 0; r < 3; r++) outp[no][r] = P[r] + t * (Q[r] - P[r]);
          no++;
        }
      }
      np = no;
      std::memcpy(poly, outp, sizeof(double) * 3 * no);
    }
    double nout[3] = {refA ? nr[0] : -nr[0], refA ? nr[1] : -nr[1], refA ? nr[2] : -nr[2]};
    for (int q = 0; q < np; q++) {
      double dq[3] = {poly[q][0] - cR[0], poly[q][1] - cR[1], poly[q][2] - cR[2]};
      double depth = dot3(nr, dq);
      if (depth < 0) {
        Contact c = proto;
        c.dist = depth;
        for (int r = 0; r < 3; r++) c.pos[r] = poly[q][r] - 0.5 * depth * nr[r];
        contact_frame(nout, c.frame);
        out.push_back(c);
      }
    }
  } else {
    int i = (best - 6) / 3, j = (best - 6) % 3;
    double n[3] = {L[best][0], L[best][1], L[best][2]};
    if (dot3(n, d) < 0) for (int r = 0; r < 3; r++) n[r] = -n[r];
    double pA[3] = {cA[0], cA[1], cA[2]}, pB[3] = {cB[0], cB[1], cB[2]};
    for (int k = 0; k < 3; k++) {
      if (k != i) { double sg = dot3(a[k], n) >= 0 ? 1.0 : -1.0; for (int r = 0; r < 3; r++) pA[r] += sg * hA[k] * a[k][r]; }
      if (k != j) { double sg = dot3(b[k], n) >= 0 ? 1.0 : -1.0; for (int r = 0; r < 3; r++) pB[r] -= sg * hB[k] * b[k][r]; }
    }
    double w0[3] = {pA[0] - pB[0], pA[1] - pB[1], pA[2] - pB[2]};
    double bb = dot3(a[i], b[j]), dd = dot3(a[i], w0), ee = dot3(b[j], w0), den = 1 - bb * bb;
    double sp = den > 1e-12 ? (bb * ee - dd) / den : 0.0;
    double tp = ee + sp * bb;
    sp = std::max(-hA[i], std::min(hA[i], sp));
    tp = std::max(-hB[j], std::min(hB[j], tp));
    Contact c = proto;
    c.dist = -ov[best];
    for (int r = 0; r < 3; r++) c.pos[r] = 0.5 * (pA[r] + sp * a[i][r] + pB[r] + tp * b[j][r]);
    contact_frame(n, c.frame);
    out.push_back(c);
  }
  return (int)out.size() - n0;
}

void collide_hfield(const Model &m, const Kin &k, int g1, int g2, std::vector<Contact> &out, const Contact &proto);

// Narrow phase for one pair; geom1 is the plane for plane pairs. margin = gap = 0.
void collide_pair(const Model &m, const Kin &k, int g1, int g2, std::vector<Contact> &out) {
  Contact proto{};
  proto.g1 = g1; proto.g2 = g2; proto.b1 = m.gbody[g1]; proto.b2 = m.gbody[g2];
  proto.mu = std::max(m.gfric[g1], m.gfric[g2]);
  if (m.gtype[g1] == HFIELD) {
    collide_hfield(m, k, g1, g2, out, proto);
    return;
  }
  if (m.gtype[g1] == BOX && m.gtype[g2] == BOX) {
    box_box(&k.gxpos[3 * g1], &k.gxmat[9 * g1], &m.gsize[3 * g1], &k.gxpos[3 * g2], &k.gxmat[9 * g2],
            &m.gsize[3 * g2], out, proto, nullptr, nullptr);
    return;
  }
  const double *Rp = &k.gxmat[9 * g1];
  double n[3] = {Rp[2], Rp[5], Rp[8]};
  const double *p0 = &k.gxpos[3 * g1];
  const double *c = &k.gxpos[3 * g2];
  const double *R = &k.gxmat[9 * g2];
  const double *sz = &m.gsize[3 * g2];
  int t2 = m.gtype[g2];
  if (t2 == SPHERE) {
    plane_point(n, p0, c, sz[0], out, proto);
  } else if (t2 == CAPSULE) {
    double ax[3] = {R[2], R[5], R[8]};
    for (int e = 0; e < 2; e++) {
      double sgn = e == 0 ? -1.0 : 1.0, pe[3];
      for (int i = 0; i < 3; i++) pe[i] = c[i] + sgn * sz[1] * ax[i];
      plane_point(n, p0, pe, sz[0], out, proto);
    }
  } else if (t2 == BOX) {
    // every vertex below the plane; keep the 4 deepest (lower vertex index on ties)
    double depth[8], vert[8][3];
    int idx[8], cnt = 0;
    for (int v = 0; v < 8; v++) {
      double loc[3] = {(v & 1 ? 1.0 : -1.0) * sz[0], (v & 2 ? 1.0 : -1.0) * sz[1],
                       (v & 4 ? 1.0 : -1.0) * sz[2]};
      double w[3];
      matvec3(R, loc, w);
      for (int i = 0; i < 3; i++) vert[v][i] = c[i] + w[i];
      double diff[3] = {vert[v][0] - p0[0], vert[v][1] - p0[1], vert[v][2] - p0[2]};
      depth[v] = dot3(n, diff);
      if (depth[v] < 0) idx[cnt++] = v;
    }
    // selection of the 4 deepest by (depth, index), then back to index order
    for (int a = 0; a < cnt; a++)
      for (int b = a + 1; b < cnt; b++)
        if (depth[idx[b]] < depth[idx[a]] || (depth[idx[b]] == depth[idx[a]] && idx[b] < idx[a])) {
          int t = idx[a]; idx[a] = idx[b]; idx[b] = t;
        }
    cnt = cnt < 4 ? cnt : 4;
    for (int a = 0; a < cnt; a++)
      for (int b = a + 1; b < cnt; b++)
        if (idx[b] < idx[a]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    for (int q = 0; q < cnt; q++) {
      int v = idx[q];
      Contact cc = proto;
      cc.dist = depth[v];
      for (int i = 0; i < 3; i++) cc.pos[i] = vert[v][i] - 0.5 * depth[v] * n[i];
      contact_frame(n, cc.frame);
      out.push_back(cc);
    }
  }
}

// ------------------------------------------------------------------ heightfield
// The elevation grid spans [-hx, hx] x [-hy, hy] in the geom frame with ncol x nrow
// samples; each cell (i, j) is split along its (i, j)-(i+1, j+1) diagonal into the
// triangles (v00, v10, v11) and (v00, v11, v01); the solid lies below the surface and
// there is no terrain outside the grid (reading of MuJoCo's heightfield as a triangle
// surface).
struct HTri { double v[3][3], n[3]; };
void hf_vertex(const Model &m, int i, int j, double *v) {
  double dx = 2 * m.hf_size[0] / (m.hf_ncol - 1), dy = 2 * m.hf_size[1] / (m.hf_nrow - 1);
  v[0] = -m.hf_size[0] + j * dx;
  v[1] = -m.hf_size[1] + i * dy;
  v[2] = m.hf[(size_t)i * m.hf_ncol + j];
}
HTri hf_triangle(const Model &m, int i, int j, int upper) {
  HTri t;
  double v00[3], v10[3], v11[3], v01[3];
  hf_vertex(m, i, j, v00); hf_vertex(m, i, j + 1, v10); hf_vertex(m, i + 1, j + 1, v11); hf_vertex(m, i + 1, j, v01);
  const double *a = v00, *b = upper ? v11 : v10, *c = upper ? v01 : v11;
  for (int k = 0; k < 3; k++) { t.v[0][k] = a[k]; t.v[1][k] = b[k]; t.v[2][k] = c[k]; }
  double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  cross3(e1, e2, t.n);
  double l = std::sqrt(dot3(t.n, t.n));
  for (int k = 0; k < 3; k++) t.n[k] /= l;
  return t;
}
// cell and triangle under the point (x, y); false outside the grid
bool hf_locate(const Model &m, double x, double y, int &i, int &j, int &upper) {
  double dx = 2 * m.hf_size[0] / (m.hf_ncol - 1), dy = 2 * m.hf_size[1] / (m.hf_nrow - 1);
  double u = (x + m.hf_size[0]) / dx, v = (y + m.hf_size[1]) / dy;
  if (u < 0 || v < 0 || u > m.hf_ncol - 1 || v > m.hf_nrow - 1) return false;
  j = std::min((int)u, m.hf_ncol - 2);
  i = std::min((int)v, m.hf_nrow - 2);
  upper = (v - i) > (u - j) ? 1 : 0;
  return true;
}
// closest point of a triangle to p (Voronoi regions of the vertices, edges and face)
void closest_on_triangle(const double *p, const HTri &t, double *q) {
  const double *a = t.v[0], *b = t.v[1], *c = t.v[2];
  double ab[3], ac[3], ap[3];
  for (int k = 0; k < 3; k++) { ab[k] = b[k] - a[k]; ac[k] = c[k] - a[k]; ap[k] = p[k] - a[k]; }
  double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
  if (d1 <= 0 && d2 <= 0) { for (int k = 0; k < 3; k++) q[k] = a[k]; return; }
  double bp[3] = {p[0] - b[0], p[1] - b[1], p[2] - b[2]};
  double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
  if (d3 >= 0 && d4 <= d3) { for (int k = 0; k < 3; k++) q[k] = b[k]; return; }
  double vc = d1 * d4 - d3 * d2;
  if (vc <= 0 && d1 >= 0 && d3 <= 0) {
    double s = d1 / (d1 - d3);
    for (int k = 0; k < 3; k++) q[k] = a[k] + s * ab[k];
    return;
  }
  double cp[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
  double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
  if (d6 >= 0 && d5 <= d6) { for (int k = 0; k < 3; k++) q[k] = c[k]; return; }
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0 && d2 >= 0 && d6 <= 0) {
    double s = d2 / (d2 - d6);
    for (int k = 0; k < 3; k++) q[k] = a[k] + s * ac[k];
    return;
  }
  double va = d3 * d6 - d5 * d4;
  if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
    double s = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    for (int k = 0; k < 3; k++) q[k] = b[k] + s * (c[k] - b[k]);
    return;
  }
  double den = 1.0 / (va + vb + vc), v = vb * den, w = vc * den;
  for (int k = 0; k < 3; k++) q[k] = a[k] + v * ab[k] + w * ac[k];
}
// a sphere (centre c, radius r, geom frame) against the surface: centre below the surface
// under it -> that triangle's normal and signed distance; else the closest surface point
// over the cells the sphere's footprint covers. Returns false without contact.
bool hf_sphere(const Model &m, const double *c, double r, double *n, double *dist) {
  int i, j, up;
  if (!hf_locate(m, c[0], c[1], i, j, up)) return false;
  HTri t = hf_triangle(m, i, j, up);
  double d0[3] = {c[0] - t.v[0][0], c[1] - t.v[0][1], c[2] - t.v[0][2]};
  double sd = dot3(t.n, d0);
  if (sd < 0) {
    for (int k = 0; k < 3; k++) n[k] = t.n[k];
    *dist = sd - r;
    return true;
  }
  double dx = 2 * m.hf_size[0] / (m.hf_ncol - 1), dy = 2 * m.hf_size[1] / (m.hf_nrow - 1);
  int j0 = std::max(0, (int)std::floor((c[0] - r + m.hf_size[0]) / dx));
  int j1 = std::min(m.hf_ncol - 2, (int)std::floor((c[0] + r + m.hf_size[0]) / dx));
  int i0 = std::max(0, (int)std::floor((c[1] - r + m.hf_size[1]) / dy));
  int i1 = std::min(m.hf_nrow - 2, (int)std::floor((c[1] + r + m.hf_size[1]) / dy));
  double best = 1e300, bq[3] = {0, 0, 0};
  for (int ii = i0; ii <= i1; ii++)
    for (int jj = j0; jj <= j1; jj++)
      for (int u = 0; u < 2; u++) {
        HTri tt = hf_triangle(m, ii, jj, u);
        double q[3];
        closest_on_triangle(c, tt, q);
        double e[3] = {c[0] - q[0], c[1] - q[1], c[2] - q[2]};
        double l2 = dot3(e, e);
        if (l2 < best) { best = l2; for (int k = 0; k < 3; k++) bq[k] = q[k]; }
      }
  double l = std::sqrt(best);
  if (!(l < r) || l <= 0) return false;
  for (int k = 0; k < 3; k++) n[k] = (c[k] - bq[k]) / l;
  *dist = l - r;
  return true;
}

// heightfield (geom1) against a sphere, capsule end spheres or box vertices (geom2);
// every contact has its own normal (world frame) and the midpoint position
void collide_hfield(const Model &m, const Kin &k, int g1, int g2, std::vector<Contact> &out, const Contact &proto) {
  const double *hc = &k.gxpos[3 * g1], *HR = &k.gxmat[9 * g1];
  const double *c = &k.gxpos[3 * g2], *R = &k.gxmat[9 * g2], *sz = &m.gsize[3 * g2];
  auto to_local = [&](const double *pw, double *pl) {
    double d[3] = {pw[0] - hc[0], pw[1] - hc[1], pw[2] - hc[2]};
    for (int a = 0; a < 3; a++) pl[a] = HR[a] * d[0] + HR[3 + a] * d[1] + HR[6 + a] * d[2];
  };
  auto emit = [&](const double *cw, double r, const double *nl, double dist) {
    Contact cc = proto;
    double nw[3];
    matvec3(HR, nl, nw);
    cc.dist = dist;
    for (int a = 0; a < 3; a++) cc.pos[a] = cw[a] - nw[a] * (r + 0.5 * dist);
    contact_frame(nw, cc.frame);
    out.push_back(cc);
  };
  int t2 = m.gtype[g2];
  if (t2 == SPHERE || t2 == CAPSULE) {
    int ne = t2 == SPHERE ? 1 : 2;
    for (int e = 0; e < ne; e++) {
      double sg = t2 == SPHERE ? 0.0 : (e == 0 ? -sz[1] : sz[1]);
      double pw[3] = {c[0] + sg * R[2], c[1] + sg * R[5], c[2] + sg * R[8]}, pl[3], nl[3], dist;
      to_local(pw, pl);
      if (hf_sphere(m, pl, sz[0], nl, &dist)) emit(pw, sz[0], nl, dist);
    }
  } else if (t2 == BOX) {
    // candidates: (a) box vertices below the surface (depth along the normal of the triangle
    // under them), (b) convex grid vertices inside the box (depth = minus the distance to the
    // nearest box face; normal = the inward normal of that face, pointing from the terrain
    // into the box). The four deepest are kept (ties: box vertices by index, then grid
    // vertices in row-major order) and emitted in that candidate order.
    struct Cand { double depth; long key; double pos[3], n[3]; };
    std::vector<Cand> cand;
    double vw[8][3], ploc[8][3];
    for (int v = 0; v < 8; v++) {
      double loc[3] = {(v & 1 ? 1.0 : -1.0) * sz[0], (v & 2 ? 1.0 : -1.0) * sz[1], (v & 4 ? 1.0 : -1.0) * sz[2]};
      double w[3];
      matvec3(R, loc, w);
      for (int a = 0; a < 3; a++) vw[v][a] = c[a] + w[a];
      to_local(vw[v], ploc[v]);
      int i, j, up;
      if (hf_locate(m, ploc[v][0], ploc[v][1], i, j, up)) {
        HTri t = hf_triangle(m, i, j, up);
        double d0[3] = {ploc[v][0] - t.v[0][0], ploc[v][1] - t.v[0][1], ploc[v][2] - t.v[0][2]};
        double dep = dot3(t.n, d0);
        if (dep < 0) {
          Cand k{dep, v, {0, 0, 0}, {0, 0, 0}};
          double nw[3];
          matvec3(HR, t.n, nw);
          for (int a = 0; a < 3; a++) { k.n[a] = nw[a]; k.pos[a] = vw[v][a] - nw[a] * 0.5 * dep; }
          cand.push_back(k);
        }
      }
    }
    // grid vertices under the box's footprint (grid frame)
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int v = 0; v < 8; v++) {
      xmin = std::min(xmin, ploc[v][0]); xmax = std::max(xmax, ploc[v][0]);
      ymin = std::min(ymin, ploc[v][1]); ymax = std::max(ymax, ploc[v][1]);
    }
    double dx = 2 * m.hf_size[0] / (m.hf_ncol - 1), dy = 2 * m.hf_size[1] / (m.hf_nrow - 1);
    int j0 = std::max(0, (int)std::ceil((xmin + m.hf_size[0]) / dx)), j1 = std::min(m.hf_ncol - 1, (int)std::floor((xmax + m.hf_size[0]) / dx));
    int i0 = std::max(0, (int)std::ceil((ymin + m.hf_size[1]) / dy)), i1 = std::min(m.hf_nrow - 1, (int)std::floor((ymax + m.hf_size[1]) / dy));
    for (int i = i0; i <= i1; i++)
      for (int j = j0; j <= j1; j++) {
        if (!m.hf_convex[(size_t)i * m.hf_ncol + j]) continue;
        double gl[3], gw[3], dpos[3], p[3];
        hf_vertex(m, i, j, gl);
        matvec3(HR, gl, gw);
        for (int a = 0; a < 3; a++) { gw[a] += hc[a]; dpos[a] = gw[a] - c[a]; }
        for (int a = 0; a < 3; a++) p[a] = R[a] * dpos[0] + R[3 + a] * dpos[1] + R[6 + a] * dpos[2];  // box frame
        if (!(std::fabs(p[0]) < sz[0] && std::fabs(p[1]) < sz[1] && std::fabs(p[2]) < sz[2])) continue;
        int kf = 0;
        double best = sz[0] - std::fabs(p[0]);
        for (int a = 1; a < 3; a++)
          if (sz[a] - std::fabs(p[a]) < best) { best = sz[a] - std::fabs(p[a]); kf = a; }
        double fl[3] = {0, 0, 0};
        fl[kf] = p[kf] >= 0 ? -1.0 : 1.0;          // inward normal of the nearest face (box frame)
        Cand k{-best, 8 + (long)i * m.hf_ncol + j, {0, 0, 0}, {0, 0, 0}};
        matvec3(R, fl, k.n);
        for (int a = 0; a < 3; a++) k.pos[a] = gw[a] + k.n[a] * 0.5 * k.depth;
        cand.push_back(k);
      }
    std::sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) {
      return x.depth < y.depth || (x.depth == y.depth && x.key < y.key);
    });
    if (cand.size() > 4) cand.resize(4);
    std::sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.key < y.key; });
    for (const Cand &k : cand) {
      Contact cc = proto;
      cc.dist = k.depth;
      for (int a = 0; a < 3; a++) cc.pos[a] = k.pos[a];
      contact_frame(k.n, cc.frame);
      out.push_back(cc);
    }
  }
}

int collide_all(const Model &m, const Kin &k, std::vector<Contact> &out, int cap, bool *overflow) {
  out.clear();
  for (size_t p = 0; p < m.pairs.size() / 2; p++) collide_pair(m, k, m.pairs[2 * p], m.pairs[2 * p + 1], out);
  *overflow = (int)out.size() > cap;
  if (*overflow) out.resize(cap);
  return (int)out.size();
}

// ------------------------------------------------------------------ constraint model
// Impedance d(r) (MuJoCo solimp = dmin, dmax, width, midpoint, power), clamped to
// [1e-4, 0.9999].
double impedance(const Model &m, double r) {
  double dmin = m.solimp[0], dmax = m.solimp[1], width = m.solimp[2], mid = m.solimp[3], pw = m.solimp[4];
  double x = std::fabs(r) / width, d;
  if (!(width > 0) || x >= 1) {
    d = dmax;
  } else {
    double y = x <= mid ? std::pow(x, pw) / std::pow(mid, pw - 1)
                        : 1 - std::pow(1 - x, pw) / std::pow(1 - mid, pw - 1);
    d = dmin + y * (dmax - dmin);
  }
  return std::min(0.9999, std::max(1e-4, d));
}

// point Jacobian column (translational velocity of a point p fixed to the moving
// body, per unit qvel_d): lin + ang x p for spatial vectors about O.
void point_jac(const Model &m, const Kin &k, int b, const double *p, double *Jp /*3 x nv*/) {
  for (int d = 0; d < m.nv; d++) {
    double col[3] = {0, 0, 0};
    if (b > 0 && dof_moves(m, d, b)) {
      const double *s = &k.cdof[6 * d];
      cross3(s, p, col);
      for (int i = 0; i < 3; i++) col[i] += s[3 + i];
    }
    for (int i = 0; i < 3; i++) Jp[i * m.nv + d] = col[i];
  }
}

// rows (normal, t1, t2) = frame (J_p(b2) - J_p(b1)); aref = -b J qvel - k d r (r = dist on
// the normal row, 0 on tangent rows); R = max(1e-15, (1-d)/d A_nn), A_nn = j_n M^-1 j_n^T,
// shared by the three rows of a contact (isotropic elliptic cone).
struct Rows {
  int nc = 0;
  std::vector<double> J, aref, R, D, mu;
};
void build_rows(const Model &m, const Kin &k, const std::vector<Contact> &con, const double *qvel,
                const std::vector<double> &ML, const std::vector<double> &MD, double friction_scale,
                Rows &rows) {
  int nv = m.nv, nc = (int)con.size();
  rows.nc = nc;
  rows.J.assign(3 * nc * nv, 0.0);
  rows.aref.assign(3 * nc, 0.0);
  rows.R.assign(3 * nc, 0.0);
  rows.D.assign(3 * nc, 0.0);
  rows.mu.assign(nc, 0.0);
  double tc = std::max(m.solref[0], 2 * m.h), zeta = m.solref[1], dmax = m.solimp[1];
  double B = 2 / (dmax * tc), K = 1 / (dmax * dmax * tc * tc * zeta * zeta);
  std::vector<double> J1(3 * nv), J2(3 * nv), x(nv);
  for (int c = 0; c < nc; c++) {
    const Contact &cc = con[c];
    point_jac(m, k, cc.b1, cc.pos, J1.data());
    point_jac(m, k, cc.b2, cc.pos, J2.data());
    for (int r = 0; r < 3; r++)
      for (int d = 0; d < nv; d++) {
        double s = 0;
        for (int i = 0; i < 3; i++) s += cc.frame[3 * r + i] * (J2[i * nv + d] - J1[i * nv + d]);
        rows.J[(3 * c + r) * nv + d] = s;
      }
    double dimp = impedance(m, cc.dist);
    for (int d = 0; d < nv; d++) x[d] = rows.J[(3 * c) * nv + d];
    dense_ldl_solve(nv, ML, MD, x.data());
    double A = 0;
    for (int d = 0; d < nv; d++) A += rows.J[(3 * c) * nv + d] * x[d];
    double R = std::max(1e-15, (1 - dimp) / dimp * A);
    for (int r = 0; r < 3; r++) {
      double vel = 0;
      for (int d = 0; d < nv; d++) vel += rows.J[(3 * c + r) * nv + d] * qvel[d];
      double pos = r == 0 ? cc.dist : 0.0;
      rows.aref[3 * c + r] = -B * vel - K * dimp * pos;
      rows.R[3 * c + r] = R;
      rows.D[3 * c + r] = 1 / R;
    }
    rows.mu[c] = cc.mu * friction_scale;
  }
}

// Elliptic-cone cost of one contact on jar = J a - aref = (N, T1, T2):
// s = D/2 |P_K(-jar)|^2, K = {|f_t| <= mu f_n}: zero above the polar cone (mu T <= N),
// D/2 |jar|^2 inside -K (T <= -mu N), D (mu T - N)^2 / (2 (1 + mu^2)) between.
// Returns s; writes grad = ds/djar and the 3x3 Hessian.
double cone_cost(const double *jar, double mu, double D, double *grad, double *hess) {
  double N = jar[0], T = std::sqrt(jar[1] * jar[1] + jar[2] * jar[2]);
  std::fill(grad, grad + 3, 0.0);
  if (hess) std::fill(hess, hess + 9, 0.0);
  if (mu * T <= N) return 0.0;
  if (T <= -mu * N) {
    for (int i = 0; i < 3; i++) grad[i] = D * jar[i];
    if (hess) hess[0] = hess[4] = hess[8] = D;
    return 0.5 * D * (N * N + T * T);
  }
  double h = mu * T - N, c = D / (2 * (1 + mu * mu));
  double that[2] = {T > 0 ? jar[1] / T : 0.0, T > 0 ? jar[2] / T : 0.0};
  double gh[3] = {-1, mu * that[0], mu * that[1]};
  for (int i = 0; i < 3; i++) grad[i] = 2 * c * h * gh[i];
  if (hess) {
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) hess[3 * i + j] = 2 * c * gh[i] * gh[j];
    if (mu > 0 && T > 0) {
      double w = 2 * c * h * mu / T;
      for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) hess[3 * (1 + i) + 1 + j] += w * ((i == j ? 1 : 0) - that[i] * that[j]);
    }
  }
  return c * h * h;
}

// Joint limits (MuJoCo's limit constraint, read for this model): a limited hinge or
// slide joint with range [lo, hi] gets one row when violated -- q < lo: J = e_d,
// r = q - lo; q > hi: J = -e_d, r = hi - q (margin 0). Impedance, reference and
// regulariser as for a contact normal row: aref = -b J qvel - k d(r) r,
// R = max(1e-15, (1 - d)/d A), A = e_d^T M^-1 e_d; D = 1/R.
struct Limits {
  int nl = 0;
  std::vector<int> dof;
  std::vector<double> sign, dist, J, aref, R, D;
};
void build_limits(const Model &m, const double *qpos, const double *qvel, const std::vector<double> &ML,
                  const std::vector<double> &MD, Limits &L) {
  int nv = m.nv;
  L = Limits();
  double tc = std::max(m.solref[0], 2 * m.h), zeta = m.solref[1], dmax = m.solimp[1];
  double B = 2 / (dmax * tc), K = 1 / (dmax * dmax * tc * tc * zeta * zeta);
  std::vector<double> x(nv);
  for (int j = 0; j < m.nj; j++) {
    if (m.jlimited.empty() || !m.jlimited[j] || m.jtype[j] == FREE) continue;
    double q = qpos[m.qadr[j]], lo = m.jrange[2 * j], hi = m.jrange[2 * j + 1];
    double sg, r;
    if (q - lo < 0) { sg = 1; r = q - lo; }
    else if (hi - q < 0) { sg = -1; r = hi - q; }
    else continue;
    int d = m.dadr[j];
    std::fill(x.begin(), x.end(), 0.0);
    x[d] = 1;
    dense_ldl_solve(nv, ML, MD, x.data());
    double A = x[d];
    double dimp = impedance(m, r);
    double R = std::max(1e-15, (1 - dimp) / dimp * A);
    L.dof.push_back(d);
    L.sign.push_back(sg);
    L.dist.push_back(r);
    std::vector<double> row(nv, 0.0);
    row[d] = sg;
    L.J.insert(L.J.end(), row.begin(), row.end());
    L.aref.push_back(-B * sg * qvel[d] - K * dimp * r);
    L.R.push_back(R);
    L.D.push_back(1 / R);
    L.nl++;
  }
}

// one-sided quadratic of a limit row on x = J a - aref: D/2 min(x, 0)^2
inline double limit_cost(double x, double D, double *grad, double *hess) {
  if (x >= 0) { *grad = 0; if (hess) *hess = 0; return 0.0; }
  *grad = D * x;
  if (hess) *hess = D;
  return 0.5 * D * x * x;
}

// total cost 1/2 (a-a_s)^T M (a-a_s) + sum_c s_c(J_c a - aref_c) + sum_l D_l/2 min(J_l a - aref_l, 0)^2
double total_cost(int nv, const double *M, const double *as, int nc, const double *J, const double *aref,
                  const double *D, const double *mu, int nl, const double *Jl, const double *arefl,
                  const double *Dl, const double *a) {
  std::vector<double> e(nv);
  for (int i = 0; i < nv; i++) e[i] = a[i] - as[i];
  double q = 0;
  for (int i = 0; i < nv; i++)
    for (int j = 0; j < nv; j++) q += e[i] * M[i * nv + j] * e[j];
  double s = 0.5 * q;
  for (int c = 0; c < nc; c++) {
    double jar[3], g[3];
    for (int r = 0; r < 3; r++) {
      double v = 0;
      for (int d = 0; d < nv; d++) v += J[(3 * c + r) * nv + d] * a[d];
      jar[r] = v - aref[3 * c + r];
    }
    s += cone_cost(jar, mu[c], D[3 * c], g, nullptr);
  }
  for (int l = 0; l < nl; l++) {
    double v = 0, g;
    for (int d = 0; d < nv; d++) v += Jl[l * nv + d] * a[d];
    s += limit_cost(v - arefl[l], Dl[l], &g, nullptr);
  }
  return s;
}

// Newton's method on the convex cost with exact line search, run to convergence.
int newton(int nv, const double *M, const double *as, int nc, const double *J, const double *aref,
           const double *D, const double *mu, int nl, const double *Jl, const double *arefl, const double *Dl,
           const double *a0, double *a, double *force, double *lforce, int maxiter) {
  int nr = 3 * nc;
  double tr = 0;
  for (int i = 0; i < nv; i++) tr += M[i * nv + i];
  double scale = tr > 0 ? 1.0 / tr : 1.0;
  // warm start: the lower-cost of a0 and a_s
  std::copy(as, as + nv, a);
  if (a0 && total_cost(nv, M, as, nc, J, aref, D, mu, nl, Jl, arefl, Dl, a0) <
                total_cost(nv, M, as, nc, J, aref, D, mu, nl, Jl, arefl, Dl, as))
    std::copy(a0, a0 + nv, a);
  std::vector<double> jar(nr), g(nv), H(nv * nv), p(nv), jv(nr), Mp(nv), L, Dg, Me(nv), xl(nl), jvl(nl);
  int it = 0;
  for (; it < maxiter; it++) {
    for (int r = 0; r < nr; r++) {
      double v = 0;
      for (int d = 0; d < nv; d++) v += J[r * nv + d] * a[d];
      jar[r] = v - aref[r];
    }
    for (int i = 0; i < nv; i++) {
      double s = 0;
      for (int j = 0; j < nv; j++) s += M[i * nv + j] * (a[j] - as[j]);
      Me[i] = s;
    }
    std::copy(M, M + nv * nv, H.begin());
    std::copy(Me.begin(), Me.end(), g.begin());
    for (int c = 0; c < nc; c++) {
      double gr[3], hs[9];
      cone_cost(&jar[3 * c], mu[c], D[3 * c], gr, hs);
      for (int d = 0; d < nv; d++)
        for (int r = 0; r < 3; r++) g[d] += J[(3 * c + r) * nv + d] * gr[r];
      for (int i = 0; i < nv; i++)
        for (int j = 0; j < nv; j++) {
          double s = 0;
          for (int r = 0; r < 3; r++)
            for (int q = 0; q < 3; q++) s += J[(3 * c + r) * nv + i] * hs[3 * r + q] * J[(3 * c + q) * nv + j];
          H[i * nv + j] += s;
        }
    }
    for (int l = 0; l < nl; l++) {
      double v = 0, gr, hs;
      for (int d = 0; d < nv; d++) v += Jl[l * nv + d] * a[d];
      xl[l] = v - arefl[l];
      limit_cost(xl[l], Dl[l], &gr, &hs);
      for (int i = 0; i < nv; i++) {
        g[i] += Jl[l * nv + i] * gr;
        for (int j = 0; j < nv; j++) H[i * nv + j] += Jl[l * nv + i] * hs * Jl[l * nv + j];
      }
    }
    double gn = 0;
    for (int i = 0; i < nv; i++) gn += g[i] * g[i];
    if (scale * std::sqrt(gn) < 1e-14) break;
    if (!dense_ldl(nv, H.data(), L, Dg)) break;
    for (int i = 0; i < nv; i++) p[i] = -g[i];
    dense_ldl_solve(nv, L, Dg, p.data());
    // exact line search on phi(alpha) = cost(a + alpha p): phi is convex, C^1
    for (int r = 0; r < nr; r++) {
      double v = 0;
      for (int d = 0; d < nv; d++) v += J[r * nv + d] * p[d];
      jv[r] = v;
    }
    for (int l = 0; l < nl; l++) {
      double v = 0;
      for (int d = 0; d < nv; d++) v += Jl[l * nv + d] * p[d];
      jvl[l] = v;
    }
    double pMp = 0, pMe = 0;
    for (int i = 0; i < nv; i++) {
      double s = 0;
      for (int j = 0; j < nv; j++) s += M[i * nv + j] * p[j];
      Mp[i] = s;
      pMp += p[i] * s;
      pMe += p[i] * Me[i];
    }
    auto dphi = [&](double al, double *d2) {
      double d1 = pMe + al * pMp;
      double dd = pMp;
      for (int c = 0; c < nc; c++) {
        double x[3], gr[3], hs[9];
        for (int r = 0; r < 3; r++) x[r] = jar[3 * c + r] + al * jv[3 * c + r];
        cone_cost(x, mu[c], D[3 * c], gr, hs);
        for (int r = 0; r < 3; r++) {
          d1 += gr[r] * jv[3 * c + r];
          for (int q = 0; q < 3; q++) dd += jv[3 * c + r] * hs[3 * r + q] * jv[3 * c + q];
        }
      }
      for (int l = 0; l < nl; l++) {
        double gr, hs;
        limit_cost(xl[l] + al * jvl[l], Dl[l], &gr, &hs);
        d1 += gr * jvl[l];
        dd += hs * jvl[l] * jvl[l];
      }
      if (d2) *d2 = dd;
      return d1;
    };
    double d0 = dphi(0, nullptr);
    if (!(d0 < 0)) break;
    double lo = 0, hi = 1;
    while (dphi(hi, nullptr) < 0 && hi < 1e12) { lo = hi; hi *= 2; }
    double al = std::min(1.0, hi), d2;
    for (int ls = 0; ls < 200; ls++) {
      double d1 = dphi(al, &d2);
      if (std::fabs(d1) <= 1e-15 * std::fabs(d0)) break;
      if (d1 < 0) lo = al; else hi = al;
      if (hi - lo <= 1e-16 * hi) break;
      double an = d2 > 0 ? al - d1 / d2 : 0.5 * (lo + hi);
      if (!(an > lo && an < hi)) an = 0.5 * (lo + hi);
      al = an;
    }
    double c_old = total_cost(nv, M, as, nc, J, aref, D, mu, nl, Jl, arefl, Dl, a);
    for (int i = 0; i < nv; i++) a[i] += al * p[i];
    double c_new = total_cost(nv, M, as, nc, J, aref, D, mu, nl, Jl, arefl, Dl, a);
    if (scale * (c_old - c_new) < 1e-20) { it++; break; }
  }
  if (force) {
    for (int c = 0; c < nc; c++) {
      double x[3], gr[3];
      for (int r = 0; r < 3; r++) {
        double v = 0;
        for (int d = 0; d < nv; d++) v += J[(3 * c + r) * nv + d] * a[d];
        x[r] = v - aref[3 * c + r];
      }
      cone_cost(x, mu[c], D[3 * c], gr, nullptr);
      for (int r = 0; r < 3; r++) force[3 * c + r] = -gr[r];
    }
  }
  if (lforce) {
    for (int l = 0; l < nl; l++) {
      double v = 0, gr;
      for (int d = 0; d < nv; d++) v += Jl[l * nv + d] * a[d];
      limit_cost(v - arefl[l], Dl[l], &gr, nullptr);
      lforce[l] = -gr;
    }
  }
  return it;
}

// ------------------------------------------------------------------ integration
// semi-implicit Euler: qvel += h qacc, then qpos from the new qvel. Free-joint
// orientation: q <- q (x) exp(h w/2), w the body-frame angular velocity, renormalised.
void integrate(const Model &m, double *qpos, double *qvel, const double *qacc) {
  for (int d = 0; d < m.nv; d++) qvel[d] += m.h * qacc[d];
  for (int j = 0; j < m.nj; j++) {
    double *q = qpos + m.qadr[j];
    const double *v = qvel + m.dadr[j];
    if (m.jtype[j] == FREE) {
      for (int i = 0; i < 3; i++) q[i] += m.h * v[i];
      double w = std::sqrt(v[3] * v[3] + v[4] * v[4] + v[5] * v[5]);
      if (w > 0) {
        double dq[4];
        axis_angle_quat(v + 3, w * m.h, dq);
        double out[4];
        quat_mul(q + 3, dq, out);
        std::memcpy(q + 3, out, sizeof out);
      }
      quat_normalize(q + 3);
    } else {
      q[0] += m.h * v[0];
    }
  }
}

struct Workspace {
  Kin k;
  std::vector<double> M, bias, tau, as, ML, MD;
  std::vector<Contact> con;
  Rows rows;
  Limits lim;
};

// PD position servo, optionally limited by a DC motor's torque-speed line (reading of
// the paper's "DC motor with velocity-dependent saturation", section "Components"):
// tau_max(w) = clamp(ts (1 - w/w0), 0, tl), tau_min(w) = clamp(ts (-1 - w/w0), -tl, 0),
// tau = clamp(kp (ctrl - q) - kd w, tau_min, tau_max); ts <= 0 leaves the ideal PD.
double actuator_torque(const Model &m, int u, double ctrl, double q, double w, double kp, double kd) {
  double tau = kp * (ctrl - q) - kd * w;
  if (m.dcm.empty() || !(m.dcm[3 * u] > 0)) return tau;
  double ts = m.dcm[3 * u], w0 = m.dcm[3 * u + 1], tl = m.dcm[3 * u + 2];
  double hi = std::min(std::max(ts * (1 - w / w0), 0.0), tl);
  double lo = std::max(std::min(ts * (-1 - w / w0), 0.0), -tl);
  return std::min(std::max(tau, lo), hi);
}

// one physics substep; returns status bits and the contact count / iterations
int substep(const Model &m, Workspace &w, double *qpos, double *qvel, double *qacc, const double *ctrl,
            double friction_scale, const double *mass_scale, const double *kp, const double *kd,
            int *ncon, int *iters) {
  int nv = m.nv, status = 0;
  kinematics(m, qpos, w.k);
  motion_subspace(m, w.k);
  spatial_inertia(m, mass_scale, w.k);
  w.M.assign(nv * nv, 0.0);
  mass_matrix(m, w.k, w.M.data());
  w.bias.assign(nv, 0.0);
  std::vector<double> zero(nv, 0.0);
  inverse_dynamics(m, w.k, qvel, zero.data(), true, w.bias.data());
  // PD position actuators: tau = kp (ctrl - q) - kd qdot on the actuated joint
  w.tau.assign(nv, 0.0);
  for (int u = 0; u < m.nu; u++) {
    int j = m.act_jnt[u];
    double q = qpos[m.qadr[j]], qd = qvel[m.dadr[j]];
    w.tau[m.dadr[j]] += actuator_torque(m, u, ctrl[u], q, qd, kp[u], kd[u]);
  }
  w.as.assign(nv, 0.0);
  for (int d = 0; d < nv; d++) w.as[d] = w.tau[d] - w.bias[d];
  if (!dense_ldl(nv, w.M.data(), w.ML, w.MD)) return ST_NAN;
  dense_ldl_solve(nv, w.ML, w.MD, w.as.data());
  bool overflow = false;
  int nc = collide_all(m, w.k, w.con, m.ncon_max, &overflow);
  if (overflow) status |= ST_OVERFLOW;
  *ncon = nc;
  build_limits(m, qpos, qvel, w.ML, w.MD, w.lim);
  std::vector<double> a(nv);
  if (nc == 0 && w.lim.nl == 0) {
    std::copy(w.as.begin(), w.as.end(), a.begin());
    *iters = 0;
  } else {
    build_rows(m, w.k, w.con, qvel, w.ML, w.MD, friction_scale, w.rows);
    std::vector<double> f(3 * nc);
    *iters = newton(nv, w.M.data(), w.as.data(), nc, w.rows.J.data(), w.rows.aref.data(), w.rows.D.data(),
                    w.rows.mu.data(), w.lim.nl, w.lim.J.data(), w.lim.aref.data(), w.lim.D.data(), qacc,
                    a.data(), f.data(), nullptr, 100);
    for (int c = 0; c < nc; c++)
      for (int r = 0; r < 3; r++) w.con[c].force[r] = f[3 * c + r];
  }
  std::copy(a.begin(), a.end(), qacc);
  integrate(m, qpos, qvel, qacc);
  for (int i = 0; i < m.nq; i++) if (!std::isfinite(qpos[i])) status |= ST_NAN;
  for (int i = 0; i < nv; i++) if (!std::isfinite(qvel[i]) || !std::isfinite(qacc[i])) status |= ST_NAN;
  return status;
}

void write_contacts(const std::vector<Contact> &con, double *out, int cap) {
  int n = std::min((int)con.size(), cap);
  for (int c = 0; c < n; c++) {
    double *o = out + ORC_CON_STRIDE * c;
    std::fill(o, o + ORC_CON_STRIDE, 0.0);
    const Contact &cc = con[c];
    o[0] = cc.g1; o[1] = cc.g2; o[2] = cc.b1; o[3] = cc.b2; o[4] = cc.dist;
    for (int i = 0; i < 3; i++) o[5 + i] = cc.pos[i];
    for (int i = 0; i < 9; i++) o[8 + i] = cc.frame[i];
    o[17] = cc.mu;
    for (int i = 0; i < 3; i++) o[18 + i] = cc.force[i];
    // force in world frame
    for (int i = 0; i < 3; i++) o[21 + i] = cc.frame[i] * cc.force[0] + cc.frame[3 + i] * cc.force[1] + cc.frame[6 + i] * cc.force[2];
  }
}

void push_event(const Model &m, double *qvel, int64_t step_count, uint64_t seed, int32_t world) {
  if (m.push_period <= 0 || step_count <= 0 || step_count % m.push_period != 0) return;
  if (m.nj == 0 || m.jtype[0] != FREE) return;
  uint32_t ctr[4] = {0u, (uint32_t)world, (uint32_t)PURPOSE_PUSH, (uint32_t)step_count};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  philox(ctr, key, x);
  // Box-Muller on u1 in (0, 1], u2 in [0, 1)
  double u1 = ((double)(x[0] >> 8) + 1.0) * (1.0 / 16777216.0);
  double u2 = u24(x[1]);
  double r = std::sqrt(-2.0 * std::log(u1)), th = 2.0 * M_PI * u2;
  qvel[m.dadr[0] + 0] += m.push_sigma * r * std::cos(th);
  qvel[m.dadr[0] + 1] += m.push_sigma * r * std::sin(th);
}

}  // namespace

struct orc_model {
  Model m;
};

extern "C" {

orc_model *orc_model_create(const orc_desc *d, char *err, int errlen) {
  auto fail = [&](const std::string &s) -> orc_model * {
    if (err && errlen > 0) std::snprintf(err, errlen, "%s", s.c_str());
    return nullptr;
  };
  if (!d || d->nbody < 1 || d->njnt < 0 || d->nu < 0 || d->ngeom < 0) return fail("bad sizes");
  orc_model *om = new orc_model();
  Model &m = om->m;
  m.nb = d->nbody; m.nj = d->njnt; m.nu = d->nu; m.ng = d->ngeom;
  auto cp = [](auto *src, int n, auto &dst) { dst.assign(src, src + n); };
  cp(d->body_parent, m.nb, m.parent);
  cp(d->body_pos, 3 * m.nb, m.bpos); cp(d->body_quat, 4 * m.nb, m.bquat);
  cp(d->body_mass, m.nb, m.bmass); cp(d->body_ipos, 3 * m.nb, m.bipos);
  cp(d->body_inertia, 6 * m.nb, m.binertia);
  cp(d->jnt_type, m.nj, m.jtype); cp(d->jnt_body, m.nj, m.jbody);
  cp(d->jnt_axis, 3 * m.nj, m.jaxis); cp(d->jnt_pos, 3 * m.nj, m.jpos);
  cp(d->jnt_armature, m.nj, m.jarm); cp(d->jnt_reset_noise, m.nj, m.jnoise);
  cp(d->act_jnt, m.nu, m.act_jnt); cp(d->act_kp, m.nu, m.kp); cp(d->act_kd, m.nu, m.kd);
  cp(d->geom_type, m.ng, m.gtype); cp(d->geom_body, m.ng, m.gbody);
  cp(d->geom_size, 3 * m.ng, m.gsize); cp(d->geom_pos, 3 * m.ng, m.gpos);
  cp(d->geom_quat, 4 * m.ng, m.gquat); cp(d->geom_friction, m.ng, m.gfric);
  cp(d->geom_contype, m.ng, m.ct); cp(d->geom_conaffinity, m.ng, m.ca);
  m.h = d->timestep;
  for (int i = 0; i < 3; i++) m.grav[i] = d->gravity[i];
  m.solref[0] = d->solref[0]; m.solref[1] = d->solref[1];
  for (int i = 0; i < 5; i++) m.solimp[i] = d->solimp[i];
  m.newton_iter = d->newton_iterations; m.newton_tol = d->newton_tolerance;
  m.ls_iter = d->ls_iterations; m.pivot_tau = d->pivot_tau; m.cap = d->contact_cap;
  m.push_period = d->push_period; m.push_sigma = d->push_sigma;
  if (d->jnt_limited) {
    if (!d->jnt_range) { delete om; return fail("jnt_limited needs jnt_range"); }
    cp(d->jnt_limited, m.nj, m.jlimited);
    cp(d->jnt_range, 2 * m.nj, m.jrange);
    for (int j = 0; j < m.nj; j++)
      if (m.jlimited[j] && (m.jtype[j] == FREE || !(m.jrange[2 * j] < m.jrange[2 * j + 1]))) {
        delete om;
        return fail("a limited joint is a hinge or slide with lower < upper");
      }
  }
  if (d->hfield_data) {
    if (d->hfield_nrow < 2 || d->hfield_ncol < 2 || !(d->hfield_size[0] > 0) || !(d->hfield_size[1] > 0)) {
      delete om;
      return fail("a heightfield needs at least 2 x 2 samples and positive half extents");
    }
    m.hf_nrow = d->hfield_nrow; m.hf_ncol = d->hfield_ncol;
    m.hf_size[0] = d->hfield_size[0]; m.hf_size[1] = d->hfield_size[1];
    cp(d->hfield_data, m.hf_nrow * m.hf_ncol, m.hf);
    // convex grid vertices: the surface bends down around them (height above the mean of
    // the four grid neighbours by more than 1e-9 m); planar patches have none
    m.hf_convex.assign((size_t)m.hf_nrow * m.hf_ncol, 0);
    for (int i = 1; i + 1 < m.hf_nrow; i++)
      for (int j = 1; j + 1 < m.hf_ncol; j++) {
        const double *z = m.hf.data();
        const int n = m.hf_ncol;
        double mean = 0.25 * ((z[(i - 1) * n + j] + z[(i + 1) * n + j]) + (z[i * n + j - 1] + z[i * n + j + 1]));
        m.hf_convex[(size_t)i * n + j] = z[i * n + j] - mean > 1e-9;
      }
  }
  if (d->act_dcmotor) {
    cp(d->act_dcmotor, 3 * m.nu, m.dcm);
    for (int u = 0; u < m.nu; u++)
      if (m.dcm[3 * u] > 0 && !(m.dcm[3 * u + 1] > 0 && m.dcm[3 * u + 2] > 0)) {
        delete om;
        return fail("a DC motor needs positive no-load speed and torque limit");
      }
  }
  // tree checks and dof layout
  for (int b = 1; b < m.nb; b++)
    if (m.parent[b] < 0 || m.parent[b] >= b) { delete om; return fail("body_parent must satisfy 0 <= parent < body"); }
  m.body_jnt.assign(m.nb, -1);
  m.qadr.resize(m.nj); m.dadr.resize(m.nj);
  int qa = 0, da = 0;
  for (int j = 0; j < m.nj; j++) {
    int b = m.jbody[j];
    if (b < 1 || b >= m.nb || m.body_jnt[b] >= 0) { delete om; return fail("one joint per non-world body"); }
    if (j > 0 && b <= m.jbody[j - 1]) { delete om; return fail("joints must follow body order"); }
    if (m.jtype[j] == FREE && m.parent[b] != 0) { delete om; return fail("free joint only on a child of the world"); }
    m.body_jnt[b] = j;
    m.qadr[j] = qa; m.dadr[j] = da;
    int ndof = m.jtype[j] == FREE ? 6 : 1;
    for (int i = 0; i < ndof; i++) { m.dof_body.push_back(b); m.dof_jnt.push_back(j); }
    qa += m.jtype[j] == FREE ? 7 : 1;
    da += ndof;
  }
  m.nq = qa; m.nv = da;
  cp(d->qpos_reset, m.nq, m.qpos_reset);
  // dof parent: previous dof of the same joint, else last dof of the nearest ancestor with a joint
  m.dof_parent.assign(m.nv, -1);
  for (int dd = 0; dd < m.nv; dd++) {
    int j = m.dof_jnt[dd];
    if (dd > m.dadr[j]) { m.dof_parent[dd] = dd - 1; continue; }
    int b = m.parent[m.jbody[j]];
    while (b > 0 && m.body_jnt[b] < 0) b = m.parent[b];
    if (b > 0) {
      int jj = m.body_jnt[b];
      m.dof_parent[dd] = m.dadr[jj] + (m.jtype[jj] == FREE ? 5 : 0);
    }
  }
  for (int u = 0; u < m.nu; u++)
    if (m.act_jnt[u] < 0 || m.act_jnt[u] >= m.nj || m.jtype[m.act_jnt[u]] == FREE) { delete om; return fail("actuators drive hinge or slide joints"); }
  // collision pairs from contype/conaffinity; parent-child excluded unless the parent is the world
  auto has_dofs = [&](int b) {
    while (b > 0) { if (m.body_jnt[b] >= 0) return true; b = m.parent[b]; }
    return false;
  };
  int cmax = 0;
  for (int g1 = 0; g1 < m.ng; g1++)
    for (int g2 = g1 + 1; g2 < m.ng; g2++) {
      int b1 = m.gbody[g1], b2 = m.gbody[g2];
      if (b1 == b2) continue;
      if ((b1 > 0 && m.parent[b2] == b1) || (b2 > 0 && m.parent[b1] == b2)) continue;
      if (!((m.ct[g1] & m.ca[g2]) || (m.ct[g2] & m.ca[g1]))) continue;
      if (!has_dofs(b1) && !has_dofs(b2)) continue;
      // geom1: the lower type (the plane for plane pairs); for same-type pairs the geom on
      // the world body, else the lower index
      int a = g1, b = g2;
      if (m.gtype[b] < m.gtype[a] || (m.gtype[b] == m.gtype[a] && b2 == 0 && b1 != 0)) std::swap(a, b);
      if (m.gtype[b] == HFIELD) std::swap(a, b);   // the terrain is geom1
      int ta = m.gtype[a], tb = m.gtype[b], nmax = 0;
      if (ta == HFIELD && (m.hf.empty() || m.gbody[a] != 0)) { delete om; return fail("a heightfield geom needs elevation data and sits on the world"); }
      if (ta == HFIELD && tb == SPHERE) nmax = 1;
      else if (ta == HFIELD && tb == CAPSULE) nmax = 2;
      else if (ta == HFIELD && tb == BOX) nmax = 4;
      else if (ta == PLANE && tb == SPHERE) nmax = 1;
      else if (ta == PLANE && tb == CAPSULE) nmax = 2;
      else if (ta == PLANE && tb == BOX) nmax = 4;
      else if (ta == BOX && tb == BOX) nmax = 8;
      else { delete om; return fail("unsupported geom pair (types " + std::to_string(ta) + "," + std::to_string(tb) + ")"); }
      m.pairs.push_back(a); m.pairs.push_back(b);
      cmax += nmax;
    }
  m.ncon_max = std::min(cmax, m.cap);
  return om;
}

void orc_model_destroy(orc_model *m) { delete m; }

void orc_model_info(const orc_model *om, int32_t *out) {
  const Model &m = om->m;
  out[0] = m.nq; out[1] = m.nv; out[2] = m.nu; out[3] = m.nb; out[4] = m.ng;
  out[5] = (int)m.pairs.size() / 2; out[6] = m.ncon_max;
}

void orc_model_pairs(const orc_model *om, int32_t *out) {
  for (size_t i = 0; i < om->m.pairs.size(); i++) out[i] = om->m.pairs[i];
}

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox(ctr, key, out); }

void orc_fk(const orc_model *om, const double *qpos, double *xpos, double *xquat, double *xmat,
            double *xipos, double *gxpos, double *gxmat) {
  const Model &m = om->m;
  Kin k;
  k.init(m);
  kinematics(m, qpos, k);
  if (xpos) std::copy(k.xpos.begin(), k.xpos.end(), xpos);
  if (xquat) std::copy(k.xquat.begin(), k.xquat.end(), xquat);
  if (xmat) std::copy(k.xmat.begin(), k.xmat.end(), xmat);
  if (xipos) std::copy(k.xipos.begin(), k.xipos.end(), xipos);
  if (gxpos) std::copy(k.gxpos.begin(), k.gxpos.end(), gxpos);
  if (gxmat) std::copy(k.gxmat.begin(), k.gxmat.end(), gxmat);
}

void orc_mass_matrix(const orc_model *om, const double *qpos, const double *mass_scale, double *M) {
  const Model &m = om->m;
  Kin k;
  k.init(m);
  kinematics(m, qpos, k);
  motion_subspace(m, k);
  spatial_inertia(m, mass_scale, k);
  mass_matrix(m, k, M);
}

void orc_rne(const orc_model *om, const double *qpos, const double *qvel, const double *qacc, int gravity,
             const double *mass_scale, double *tau) {
  const Model &m = om->m;
  Kin k;
  k.init(m);
  kinematics(m, qpos, k);
  motion_subspace(m, k);
  spatial_inertia(m, mass_scale, k);
  inverse_dynamics(m, k, qvel, qacc, gravity != 0, tau);
}

// Featherstone's LTDL factorisation (RBDA sec. 6.5) of a joint-space inertia matrix on
// dense storage: M = L^T D L with L unit lower-triangular, nonzero only where the
// column dof is an ancestor of the row dof. Walks the dof-parent chains from the last
// dof to the first; returns 0, or -1 on a non-positive pivot.
int orc_ltdl(const orc_model *om, const double *M, double *L, double *D) {
  const Model &m = om->m;
  int n = m.nv;
  std::vector<double> A(M, M + n * n);
  for (int k = n - 1; k >= 0; k--) {
    for (int i = m.dof_parent[k]; i >= 0; i = m.dof_parent[i]) {
      double a = A[k * n + i] / A[k * n + k];
      for (int j = i; j >= 0; j = m.dof_parent[j]) A[i * n + j] -= a * A[k * n + j];
      A[k * n + i] = a;
    }
  }
  int rc = 0;
  for (int r = 0; r < n; r++) {
    D[r] = A[r * n + r];
    if (!(D[r] > 0)) rc = -1;
    for (int c = 0; c < n; c++) L[r * n + c] = 0;
    L[r * n + r] = 1;
    for (int i = m.dof_parent[r]; i >= 0; i = m.dof_parent[i]) L[r * n + i] = A[r * n + i];
  }
  return rc;
}

// x <- M^-1 x with M = L^T D L: solve L^T y = x (leaves to root), y /= D, L x = y.
void orc_ltdl_solve(const orc_model *om, const double *L, const double *D, double *x) {
  const Model &m = om->m;
  int n = m.nv;
  for (int k = n - 1; k >= 0; k--)
    for (int i = m.dof_parent[k]; i >= 0; i = m.dof_parent[i]) x[i] -= L[k * n + i] * x[k];
  for (int k = 0; k < n; k++) x[k] /= D[k];
  for (int k = 0; k < n; k++)
    for (int i = m.dof_parent[k]; i >= 0; i = m.dof_parent[i]) x[k] -= L[k * n + i] * x[i];
}

int orc_collide(const orc_model *om, const double *qpos, double *con, int cap) {
  const Model &m = om->m;
  Kin k;
  k.init(m);
  kinematics(m, qpos, k);
  std::vector<Contact> c;
  bool ovf;
  int n = collide_all(m, k, c, cap, &ovf);
  write_contacts(c, con, cap);
  return n;
}

int orc_constraints(const orc_model *om, const double *qpos, const double *qvel, const double *mass_scale,
                    double friction_scale, double *con, int cap, double *J, double *aref, double *R, double *mu) {
  const Model &m = om->m;
  Workspace w;
  w.k.init(m);
  kinematics(m, qpos, w.k);
  motion_subspace(m, w.k);
  spatial_inertia(m, mass_scale, w.k);
  w.M.assign(m.nv * m.nv, 0.0);
  mass_matrix(m, w.k, w.M.data());
  if (!dense_ldl(m.nv, w.M.data(), w.ML, w.MD)) return -1;
  bool ovf;
  int nc = collide_all(m, w.k, w.con, cap, &ovf);
  build_rows(m, w.k, w.con, qvel, w.ML, w.MD, friction_scale, w.rows);
  if (con) write_contacts(w.con, con, cap);
  std::copy(w.rows.J.begin(), w.rows.J.end(), J);
  std::copy(w.rows.aref.begin(), w.rows.aref.end(), aref);
  std::copy(w.rows.R.begin(), w.rows.R.end(), R);
  std::copy(w.rows.mu.begin(), w.rows.mu.end(), mu);
  return nc;
}

int orc_box_box(const double *cA, const double *RA, const double *hA, const double *cB, const double *RB,
                const double *hB, double *con, int cap, int32_t *axis, double *minov) {
  std::vector<Contact> c;
  Contact proto{};
  int n = box_box(cA, RA, hA, cB, RB, hB, c, proto, axis, minov);
  write_contacts(c, con, cap);
  return std::min(n, cap);
}

int orc_limits(const orc_model *om, const double *qpos, const double *qvel, const double *mass_scale,
               int32_t *dof, double *sign, double *dist, double *aref, double *R, int cap) {
  const Model &m = om->m;
  Workspace w;
  w.k.init(m);
  kinematics(m, qpos, w.k);
  motion_subspace(m, w.k);
  spatial_inertia(m, mass_scale, w.k);
  w.M.assign(m.nv * m.nv, 0.0);
  mass_matrix(m, w.k, w.M.data());
  if (!dense_ldl(m.nv, w.M.data(), w.ML, w.MD)) return -1;
  build_limits(m, qpos, qvel, w.ML, w.MD, w.lim);
  int n = std::min(w.lim.nl, cap);
  for (int l = 0; l < n; l++) {
    dof[l] = w.lim.dof[l]; sign[l] = w.lim.sign[l]; dist[l] = w.lim.dist[l];
    aref[l] = w.lim.aref[l]; R[l] = w.lim.R[l];
  }
  return n;
}

double orc_cost(int nv, const double *M, const double *as, int nc, const double *J, const double *aref,
                const double *D, const double *mu, int nl, const double *Jl, const double *arefl,
                const double *Dl, const double *a) {
  return total_cost(nv, M, as, nc, J, aref, D, mu, nl, Jl, arefl, Dl, a);
}

int orc_newton(int nv, const double *M, const double *as, int nc, const double *J, const double *aref,
               const double *D, const double *mu, int nl, const double *Jl, const double *arefl,
               const double *Dl, const double *a_init, double *a, double *force, double *lforce, int maxiter) {
  return newton(nv, M, as, nc, J, aref, D, mu, nl, Jl, arefl, Dl, a_init, a, force, lforce, maxiter);
}

void orc_body_jacobian(const orc_model *om, const double *qpos, int32_t body, const double *p, double *Jp,
                       double *Jr) {
  const Model &m = om->m;
  Kin k;
  k.init(m);
  kinematics(m, qpos, k);
  motion_subspace(m, k);
  point_jac(m, k, body, p, Jp);
  for (int d = 0; d < m.nv; d++)
    for (int i = 0; i < 3; i++) Jr[i * m.nv + d] = (body > 0 && dof_moves(m, d, body)) ? k.cdof[6 * d + i] : 0.0;
}

// Seeded reset: qpos = qpos_reset + noise_j (2u - 1) on hinge/slide joints, u the
// (j % 4)-th Philox word of counter {j / 4, world, RESET, 0} mapped to [0, 1) with 24
// bits; free joints at their reference pose; qvel = 0.
void orc_reset(const orc_model *om, uint64_t seed, int32_t world, double *qpos, double *qvel) {
  const Model &m = om->m;
  std::copy(m.qpos_reset.begin(), m.qpos_reset.end(), qpos);
  std::fill(qvel, qvel + m.nv, 0.0);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int j = 0; j < m.nj; j++) {
    if (m.jtype[j] == FREE || !(m.jnoise[j] > 0)) continue;
    uint32_t ctr[4] = {(uint32_t)(j / 4), (uint32_t)world, (uint32_t)PURPOSE_RESET, 0u}, x[4];
    philox(ctr, key, x);
    double u = u24(x[j % 4]);
    qpos[m.qadr[j]] += m.jnoise[j] * (2.0 * u - 1.0);
  }
}

int orc_step(const orc_model *om, double *qpos, double *qvel, double *qacc, const double *ctrl,
             double friction_scale, const double *mass_scale, const double *kp, const double *kd, int nsub,
             int64_t step_count, uint64_t seed, int32_t world, double *con, int cap, int32_t *stats,
             const double *body_inertia) {
  // per-world body inertias: a copy of the model with those masses, centres and inertias
  Model local;
  if (body_inertia) {
    local = om->m;
    for (int b = 0; b < local.nb; b++) {
      const double *bi = body_inertia + 10 * (size_t)b;
      local.bmass[b] = bi[0];
      for (int i = 0; i < 3; i++) local.bipos[3 * b + i] = bi[1 + i];
      for (int i = 0; i < 6; i++) local.binertia[6 * b + i] = bi[4 + i];
    }
  }
  const Model &m = body_inertia ? local : om->m;
  Workspace w;
  w.k.init(m);
  push_event(m, qvel, step_count, seed, world);
  int status = 0, ncon = 0, iters = 0, it_sum = 0;
  for (int s = 0; s < nsub; s++) {
    status |= substep(m, w, qpos, qvel, qacc, ctrl, friction_scale, mass_scale, kp ? kp : m.kp.data(),
                      kd ? kd : m.kd.data(), &ncon, &iters);
    it_sum += iters;
    if (status & ST_NAN) break;
  }
  if (con) write_contacts(w.con, con, cap);
  if (stats) { stats[0] = ncon; stats[1] = it_sum; stats[2] = status; }
  return status;
}

int orc_step_batch(const orc_model *om, int nworld, double *qpos, double *qvel, double *qacc,
                   const double *ctrl, const double *friction_scale, const double *mass_scale,
                   const double *kp, const double *kd, int nsub, const int64_t *step_count, uint64_t seed,
                   const int32_t *world_id, int32_t *stats, int nthreads, const double *body_inertia) {
  const Model &m = om->m;
  if (nthreads < 1) nthreads = 1;
  auto work = [&](int w0, int w1) {
    for (int w = w0; w < w1; w++) {
      int32_t st[3];
      orc_step(om, qpos + (size_t)w * m.nq, qvel + (size_t)w * m.nv, qacc + (size_t)w * m.nv,
               ctrl + (size_t)w * m.nu, friction_scale ? friction_scale[w] : 1.0,
               mass_scale ? mass_scale + (size_t)w * m.nb : nullptr, kp ? kp + (size_t)w * m.nu : nullptr,
               kd ? kd + (size_t)w * m.nu : nullptr, nsub, step_count ? step_count[w] : 0, seed,
               world_id ? world_id[w] : w, nullptr, 0, st,
               body_inertia ? body_inertia + (size_t)w * 10 * m.nb : nullptr);
      if (stats) std::copy(st, st + 3, stats + 3 * (size_t)w);
    }
  };
  std::vector<std::thread> th;
  int per = (nworld + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; t++) {
    int w0 = t * per, w1 = std::min(nworld, w0 + per);
    if (w0 >= w1) break;
    th.emplace_back(work, w0, w1);
  }
  for (auto &t : th) t.join();
  return 0;
}

}  // extern "C"
