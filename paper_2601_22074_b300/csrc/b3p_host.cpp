// Host side of the b3phys C ABI: model validation and compilation into the
// device layout (dof tree, tree-sparse mass-matrix rows, body levels, collision
// pairs), batch layout inside the caller's device buffer, launches, readback,
// CUDA-graph capture. The library never allocates device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/b3phys.h"
#include "b3p_internal.h"

namespace {

thread_local std::string g_err;

b3p_status fail(b3p_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
b3p_status cuda_fail(cudaError_t e, const char *what) {
  return fail(B3P_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}
#define CUDA_TRY(x, what)                    \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

inline int pad4(int n) { return (n + 3) & ~3; }
inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

void quat_to_mat(const double *q, float *R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = std::sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  double r[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                 2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                 2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
  for (int i = 0; i < 9; i++) R[i] = (float)r[i];
}

}  // namespace

// Compiled model: derived structure kept on the host until a batch uploads it.
struct b3p_model {
  int nb = 0, nj = 0, nu = 0, ng = 0, nq = 0, nv = 0, npair = 0, ncon_max = 0, nM = 0, maxlevel = 0;
  int first_free_dof = -1;
  int newton_iter = 0, ls_iter = 0, push_period = 0;
  float h = 0, grav[3] = {0, 0, 0}, ref_b = 0, ref_k = 0, imp[5] = {0, 0, 0, 0, 0}, tol = 0, pivot_tau = 0,
        push_sigma = 0;
  // int arrays
  std::vector<int> body_parent, body_jnt, body_root, body_dl, level_body, level_start, child_start, child_list;
  std::vector<int> body_geom_adr, body_geom;   // geoms of each body (ray-cast hierarchy)
  std::vector<int> level_rec;   // packed per-body data of the level traversals
  std::vector<int> jnt_type, jnt_qadr, jnt_dadr, dof_body, dof_jnt, dof_rowadr, dof_rowlen, colind, entry_row;
  std::vector<int> col_start, col_k, col_pos, act_qadr, act_dadr, geom_type, geom_body, pair_g1, pair_g2;
  std::vector<int> sym_start;            // [nv + 1] full symmetric rows of M (M x)
  std::vector<unsigned> sym_ops;         // entry | column dof << 12, row part then column part
  std::vector<unsigned> entry_ops;       // per stored entry: row's diagonal entry | row << 12 | column << 18
  std::vector<int> ltdl_adr, chain_adr;
  std::vector<unsigned> ltdl_ops, chain_ops;
  std::vector<unsigned long long> body_mask, dof_mask;
  std::vector<int> tri_pq;
  int dense = 0;
  // float arrays
  std::vector<float> body_pos, body_quat, body_mass, body_ipos, body_inertia, jnt_axis, jnt_pos, jnt_noise;
  std::vector<float> qpos_reset, dof_armature, act_kp, act_kd, geom_size, geom_pos, geom_mat, geom_friction;
  // joint limits, DC motors, actuation delay
  std::vector<int> lim_dof, lim_qadr;
  std::vector<float> lim_range, act_dcm;
  int dcmotor = 0, act_delay = 0;
  int hf_nrow = 0, hf_ncol = 0;
  float hf_hx = 0, hf_hy = 0;
  std::vector<float> hf_data;
  std::vector<int> hf_convex;   // [nrow][ncol] 1: interior vertex above the mean of its 4 neighbours
  // shared-memory layout
  int smem_floats = 0;
  int o[28];
};

namespace {
enum {
  O_QPOS, O_QVEL, O_QACC, O_QS, O_FRC, O_CTRL, O_KP, O_KD, O_MS, O_XPOS, O_XQUAT, O_XMAT, O_CDOF, O_TMP6, O_CVEL,
  O_UNION, O_M, O_L, O_H, O_HDIAG, O_MA, O_MP, O_G, O_P, O_CON, O_CONI, O_MISC, O_LIM
};
}

struct b3p_batch {
  std::vector<const b3p_model *> models;
  std::vector<int> nworld, world_start;
  b3p_options opt{};
  char *base = nullptr;
  uint64_t bytes = 0;
  DBatch host{};
  DBatch *dev = nullptr;
  int total_world = 0, smem_floats = 0;
  uint64_t state_off = 0, state_bytes = 0;
  int wpb = 4, grid = 0, smem_bytes = 0;
  int lane_smem = 0;   // bytes per CTA of the lane solve launch (0: the solve runs one world per warp)
  int aux_smem = 0;    // bytes per CTA of the smooth launches' shared scratch (0: in the working set)
  int solve_smem = 0;  // bytes per CTA of the solve launch's Newton arrays (0: in the working set)
  int *counter = nullptr;
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_version = -1, layout_version = 0;
};

extern "C" {

const char *b3p_last_error(void) { return g_err.c_str(); }
const char *b3p_version(void) { return "b3phys 0.1 sm_103a"; }

b3p_status b3p_model_create(const b3p_model_desc *d, b3p_model **out) {
  if (!d || !out) return fail(B3P_ERR_INVALID_ARG, "null descriptor or output");
  *out = nullptr;
  if (d->nbody < 1 || d->njnt < 0 || d->nu < 0 || d->ngeom < 0) return fail(B3P_ERR_BAD_MODEL, "negative sizes");
  if (d->nbody > 1 && (!d->body_parent || !d->body_pos || !d->body_quat || !d->body_mass || !d->body_ipos ||
                       !d->body_inertia))
    return fail(B3P_ERR_INVALID_ARG, "missing body arrays");
  if (d->njnt > 0 && (!d->jnt_type || !d->jnt_body || !d->jnt_axis || !d->jnt_pos || !d->jnt_armature ||
                      !d->jnt_reset_noise || !d->qpos_reset))
    return fail(B3P_ERR_INVALID_ARG, "missing joint arrays");
  if (d->nu > 0 && (!d->act_jnt || !d->act_kp || !d->act_kd)) return fail(B3P_ERR_INVALID_ARG, "missing actuator arrays");
  if (d->ngeom > 0 && (!d->geom_type || !d->geom_body || !d->geom_size || !d->geom_pos || !d->geom_quat ||
                       !d->geom_contype || !d->geom_conaffinity || !d->geom_friction))
    return fail(B3P_ERR_INVALID_ARG, "missing geom arrays");
  if (!(d->timestep > 0)) return fail(B3P_ERR_BAD_MODEL, "timestep must be positive");
  if (d->newton_iterations < 1 || d->ls_iterations < 1) return fail(B3P_ERR_BAD_MODEL, "iteration caps must be >= 1");
  if (d->contact_cap < 0) return fail(B3P_ERR_BAD_MODEL, "negative contact cap");
  if (!(d->solimp[2] >= 0) || !(d->solimp[1] > 0) || !(d->solimp[1] < 1) || !(d->solimp[0] > 0) ||
      !(d->solimp[3] > 0 && d->solimp[3] < 1))
    return fail(B3P_ERR_BAD_MODEL, "solimp out of range");
  b3p_model *m = new b3p_model();
  auto bad = [&](b3p_status code, const char *msg) {
    delete m;
    return fail(code, "%s", msg);
  };
  m->nb = d->nbody; m->nj = d->njnt; m->nu = d->nu; m->ng = d->ngeom;
  const int nb = m->nb, nj = m->nj;
  if (nb > 64) return bad(B3P_ERR_UNSUPPORTED, "more than 64 bodies per world");
  m->body_parent.assign(nb, 0);
  for (int b = 0; b < nb; b++) m->body_parent[b] = b == 0 ? -1 : d->body_parent[b];
  for (int b = 1; b < nb; b++)
    if (m->body_parent[b] < 0 || m->body_parent[b] >= b) return bad(B3P_ERR_BAD_MODEL, "body_parent must satisfy 0 <= parent < body");
  for (int b = 0; b < nb; b++) {
    for (int k = 0; k < 3; k++) m->body_pos.push_back((float)d->body_pos[3 * b + k]);
    double q[4] = {d->body_quat[4 * b], d->body_quat[4 * b + 1], d->body_quat[4 * b + 2], d->body_quat[4 * b + 3]};
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(n > 0)) return bad(B3P_ERR_BAD_MODEL, "zero body quaternion");
    for (int k = 0; k < 4; k++) m->body_quat.push_back((float)(q[k] / n));
    if (b > 0 && !(d->body_mass[b] >= 0)) return bad(B3P_ERR_BAD_MODEL, "negative body mass");
    m->body_mass.push_back((float)d->body_mass[b]);
    for (int k = 0; k < 3; k++) m->body_ipos.push_back((float)d->body_ipos[3 * b + k]);
    for (int k = 0; k < 6; k++) m->body_inertia.push_back((float)d->body_inertia[6 * b + k]);
  }
  // joints, dofs
  m->body_jnt.assign(nb, -1);
  int qa = 0, da = 0;
  for (int j = 0; j < nj; j++) {
    int b = d->jnt_body[j], t = d->jnt_type[j];
    if (b < 1 || b >= nb || m->body_jnt[b] >= 0) return bad(B3P_ERR_BAD_MODEL, "one joint per non-world body");
    if (j > 0 && b <= d->jnt_body[j - 1]) return bad(B3P_ERR_BAD_MODEL, "joints must follow body order");
    if (t != B3P_JNT_FREE && t != B3P_JNT_HINGE && t != B3P_JNT_SLIDE) return bad(B3P_ERR_BAD_MODEL, "unknown joint type");
    if (t == B3P_JNT_FREE && m->body_parent[b] != 0) return bad(B3P_ERR_BAD_MODEL, "free joint only on a child of the world");
    m->body_jnt[b] = j;
    m->jnt_type.push_back(t);
    m->jnt_qadr.push_back(qa);
    m->jnt_dadr.push_back(da);
    double ax[3] = {d->jnt_axis[3 * j], d->jnt_axis[3 * j + 1], d->jnt_axis[3 * j + 2]};
    double an = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    if (t != B3P_JNT_FREE && !(an > 0)) return bad(B3P_ERR_BAD_MODEL, "zero joint axis");
    for (int k = 0; k < 3; k++) m->jnt_axis.push_back(t == B3P_JNT_FREE ? 0.f : (float)(ax[k] / an));
    for (int k = 0; k < 3; k++) m->jnt_pos.push_back((float)d->jnt_pos[3 * j + k]);
    m->jnt_noise.push_back((float)d->jnt_reset_noise[j]);
    int ndof = t == B3P_JNT_FREE ? 6 : 1;
    for (int k = 0; k < ndof; k++) {
      m->dof_body.push_back(b);
      m->dof_jnt.push_back(j);
      m->dof_armature.push_back(t == B3P_JNT_FREE ? 0.f : (float)d->jnt_armature[j]);
    }
    qa += t == B3P_JNT_FREE ? 7 : 1;
    da += ndof;
  }
  m->nq = qa; m->nv = da;
  for (int i = 0; i < m->nq; i++) m->qpos_reset.push_back((float)d->qpos_reset[i]);
  m->first_free_dof = (nj > 0 && m->jnt_type[0] == B3P_JNT_FREE) ? 0 : -1;
  // body roots, depths, levels, children, deepest dof on each body's chain
  std::vector<int> depth(nb, 0);
  m->body_root.assign(nb, 0);
  m->body_dl.assign(nb, -1);
  for (int b = 1; b < nb; b++) {
    int p = m->body_parent[b];
    depth[b] = depth[p] + 1;
    m->body_root[b] = p == 0 ? b : m->body_root[p];
    int j = m->body_jnt[b];
    m->body_dl[b] = j >= 0 ? m->jnt_dadr[j] + (m->jnt_type[j] == B3P_JNT_FREE ? 5 : 0) : m->body_dl[p];
  }
  m->maxlevel = 0;
  for (int b = 0; b < nb; b++) m->maxlevel = std::max(m->maxlevel, depth[b]);
  m->level_start.assign(m->maxlevel + 2, 0);
  for (int L = 0; L <= m->maxlevel; L++) {
    m->level_start[L] = (int)m->level_body.size();
    for (int b = 0; b < nb; b++) if (depth[b] == L) m->level_body.push_back(b);
  }
  m->level_start[m->maxlevel + 1] = (int)m->level_body.size();
  m->child_start.assign(nb + 1, 0);
  for (int b = 0; b < nb; b++) {
    m->child_start[b] = (int)m->child_list.size();
    for (int c = 1; c < nb; c++) if (m->body_parent[c] == b) m->child_list.push_back(c);
  }
  m->child_start[nb] = (int)m->child_list.size();
  // dof tree and tree-sparse rows: row i holds i, parent(i), parent(parent(i)), ...
  std::vector<int> dof_parent(m->nv, -1);
  for (int dd = 0; dd < m->nv; dd++) {
    int j = m->dof_jnt[dd];
    if (dd > m->jnt_dadr[j]) { dof_parent[dd] = dd - 1; continue; }
    dof_parent[dd] = m->body_dl[m->body_parent[m->dof_body[dd]]];
  }
  for (int i = 0; i < m->nv; i++) {
    m->dof_rowadr.push_back((int)m->colind.size());
    int len = 0;
    for (int k = i; k >= 0; k = dof_parent[k]) {
      m->colind.push_back(k);
      m->entry_row.push_back(i);
      len++;
    }
    if (len > B3P_MAXCHAIN) return bad(B3P_ERR_UNSUPPORTED, "a dof chain is longer than 32");
    m->dof_rowlen.push_back(len);
  }
  m->nM = (int)m->colind.size();
  // column lists: for dof i, the (row k, position) pairs of its descendants
  m->col_start.assign(m->nv + 1, 0);
  {
    std::vector<std::vector<std::pair<int, int>>> cols(m->nv);
    for (int k = 0; k < m->nv; k++)
      for (int p = 1; p < m->dof_rowlen[k]; p++) cols[m->colind[m->dof_rowadr[k] + p]].push_back({k, p});
    for (int i = 0; i < m->nv; i++) {
      m->col_start[i] = (int)m->col_k.size();
      for (auto &e : cols[i]) { m->col_k.push_back(e.first); m->col_pos.push_back(e.second); }
    }
    m->col_start[m->nv] = (int)m->col_k.size();
  }
  // full symmetric rows of M for M x: row i's stored entries (dof i and its ancestors), then
  // its descendants' entries in column i, one packed word each (entry | dof << 12)
  m->sym_start.assign(m->nv + 1, 0);
  for (int i = 0; i < m->nv; i++) {
    m->sym_start[i] = (int)m->sym_ops.size();
    for (int p = 0; p < m->dof_rowlen[i]; p++) {
      int e = m->dof_rowadr[i] + p;
      m->sym_ops.push_back((unsigned)e | (unsigned)m->colind[e] << 12);
    }
    for (int c = m->col_start[i]; c < m->col_start[i + 1]; c++) {
      int k = m->col_k[c];
      m->sym_ops.push_back((unsigned)(m->dof_rowadr[k] + m->col_pos[c]) | (unsigned)k << 12);
    }
  }
  m->sym_start[m->nv] = (int)m->sym_ops.size();
  // per stored entry, its row's diagonal entry, its row and its column in one word
  for (int e = 0; e < m->nM; e++) {
    int r = m->entry_row[e];
    m->entry_ops.push_back((unsigned)m->dof_rowadr[r] | (unsigned)r << 12 | (unsigned)m->colind[e] << 18);
  }
  // packed LTDL elimination lists and chain outer-product lists (see b3p_internal.h)
  if (m->nM > 4095) return bad(B3P_ERR_UNSUPPORTED, "more than 4095 stored mass-matrix entries");
  auto pack = [](int target, int p, int q) { return (unsigned)target | (unsigned)p << 12 | (unsigned)q << 17; };
  for (int k = 0; k < m->nv; k++) {
    int adr = m->dof_rowadr[k], len = m->dof_rowlen[k];
    m->ltdl_adr.push_back((int)m->ltdl_ops.size());
    for (int q = 1; q < len; q++)
      for (int p = 1; p <= q; p++) m->ltdl_ops.push_back(pack(m->dof_rowadr[m->colind[adr + p]] + (q - p), p, q));
    m->chain_adr.push_back((int)m->chain_ops.size());
    for (int q = 0; q < len; q++)
      for (int p = 0; p <= q; p++) m->chain_ops.push_back(pack(m->dof_rowadr[m->colind[adr + p]] + (q - p), p, q));
  }
  m->ltdl_adr.push_back((int)m->ltdl_ops.size());
  m->chain_adr.push_back((int)m->chain_ops.size());
  if (m->nv > 64) return bad(B3P_ERR_UNSUPPORTED, "more than 64 dofs per world");
  if (nb >= 4096) return bad(B3P_ERR_UNSUPPORTED, "more than 4095 bodies");
  for (int b : m->level_body) {
    int j = m->body_jnt[b], cs = m->child_start[b], nc = m->child_start[b + 1] - cs;
    if (nc > 127) return bad(B3P_ERR_UNSUPPORTED, "a body with more than 127 children");
    int jt = j >= 0 ? m->jnt_type[j] : 255, qa = j >= 0 ? m->jnt_qadr[j] : 0, da = j >= 0 ? m->jnt_dadr[j] : 0;
    m->level_rec.insert(m->level_rec.end(), {b | (m->body_parent[b] << 16), j, (jt & 0xFF) | (qa << 8),
                                             da | (cs << 12) | (nc << 24)});
  }
  m->dof_mask.assign(m->nv, 0ull);
  for (int d = 0; d < m->nv; d++)
    for (int p = 0; p < m->dof_rowlen[d]; p++) m->dof_mask[d] |= 1ull << m->colind[m->dof_rowadr[d] + p];
  m->body_mask.assign(nb, 0ull);
  for (int b = 1; b < nb; b++) {
    int dl = m->body_dl[b];
    if (dl < 0) continue;
    for (int p = 0; p < m->dof_rowlen[dl]; p++) m->body_mask[b] |= 1ull << m->colind[m->dof_rowadr[dl] + p];
  }
  // actuators
  std::vector<int> used(m->nv, 0);
  for (int u = 0; u < m->nu; u++) {
    int j = d->act_jnt[u];
    if (j < 0 || j >= nj || m->jnt_type[j] == B3P_JNT_FREE) return bad(B3P_ERR_BAD_MODEL, "actuators drive hinge or slide joints");
    if (used[m->jnt_dadr[j]]++) return bad(B3P_ERR_BAD_MODEL, "at most one actuator per joint");
    m->act_qadr.push_back(m->jnt_qadr[j]);
    m->act_dadr.push_back(m->jnt_dadr[j]);
    m->act_kp.push_back((float)d->act_kp[u]);
    m->act_kd.push_back((float)d->act_kd[u]);
    float ts = d->act_dcmotor ? (float)d->act_dcmotor[3 * u] : 0.f;
    float w0 = d->act_dcmotor ? (float)d->act_dcmotor[3 * u + 1] : 0.f;
    float tl = d->act_dcmotor ? (float)d->act_dcmotor[3 * u + 2] : 0.f;
    if (ts > 0.f && !(w0 > 0.f && tl > 0.f)) return bad(B3P_ERR_BAD_MODEL, "a DC motor needs a positive no-load speed and torque limit");
    if (ts > 0.f) m->dcmotor = 1;
    m->act_dcm.push_back(ts > 0.f ? ts : 0.f);
    m->act_dcm.push_back(w0);
    m->act_dcm.push_back(tl);
  }
  if (d->act_delay < 0 || d->act_delay > 64) return bad(B3P_ERR_BAD_MODEL, "act_delay outside 0..64");
  m->act_delay = m->nu > 0 ? d->act_delay : 0;
  // joint limits
  if (d->jnt_limited) {
    if (!d->jnt_range) return bad(B3P_ERR_INVALID_ARG, "jnt_limited needs jnt_range");
    for (int j = 0; j < nj; j++) {
      if (!d->jnt_limited[j]) continue;
      if (m->jnt_type[j] == B3P_JNT_FREE || !(d->jnt_range[2 * j] < d->jnt_range[2 * j + 1]))
        return bad(B3P_ERR_BAD_MODEL, "a limited joint is a hinge or slide with lower < upper");
      m->lim_dof.push_back(m->jnt_dadr[j]);
      m->lim_qadr.push_back(m->jnt_qadr[j]);
      m->lim_range.push_back((float)d->jnt_range[2 * j]);
      m->lim_range.push_back((float)d->jnt_range[2 * j + 1]);
    }
  }
  // geoms and pairs (same filtering rule as the descriptor documents)
  for (int g = 0; g < m->ng; g++) {
    int t = d->geom_type[g], b = d->geom_body[g];
    if (t < B3P_GEOM_PLANE || t > B3P_GEOM_HFIELD || b < 0 || b >= nb) return bad(B3P_ERR_BAD_MODEL, "bad geom type or body");
    if (t == B3P_GEOM_HFIELD && (b != 0 || !d->hfield_data))
      return bad(B3P_ERR_BAD_MODEL, "a heightfield geom sits on the world body and needs elevation data");
    m->geom_type.push_back(t);
    m->geom_body.push_back(b);
    for (int k = 0; k < 3; k++) m->geom_size.push_back((float)d->geom_size[3 * g + k]);
    for (int k = 0; k < 3; k++) m->geom_pos.push_back((float)d->geom_pos[3 * g + k]);
    float R[9];
    quat_to_mat(d->geom_quat + 4 * g, R);
    for (int k = 0; k < 9; k++) m->geom_mat.push_back(R[k]);
    m->geom_friction.push_back((float)d->geom_friction[g]);
  }
  // geoms grouped by body, in geom order within a body
  m->body_geom_adr.assign(nb + 1, 0);
  for (int b = 0; b < nb; b++) {
    m->body_geom_adr[b] = (int)m->body_geom.size();
    for (int g = 0; g < m->ng; g++)
      if (m->geom_body[g] == b) m->body_geom.push_back(g);
  }
  m->body_geom_adr[nb] = (int)m->body_geom.size();
  if (d->hfield_data) {
    if (d->hfield_nrow < 2 || d->hfield_ncol < 2 || !(d->hfield_size[0] > 0) || !(d->hfield_size[1] > 0))
      return bad(B3P_ERR_BAD_MODEL, "a heightfield needs at least 2 x 2 samples and positive half extents");
    m->hf_nrow = d->hfield_nrow; m->hf_ncol = d->hfield_ncol;
    m->hf_hx = (float)d->hfield_size[0]; m->hf_hy = (float)d->hfield_size[1];
    for (int i = 0; i < m->hf_nrow * m->hf_ncol; i++) m->hf_data.push_back((float)d->hfield_data[i]);
    // convex vertices (from the FP64 heights): the surface bends down around them by more
    // than 1e-9 m; planar patches have none. Box faces touch the terrain at these.
    m->hf_convex.assign((size_t)m->hf_nrow * m->hf_ncol, 0);
    const double *z = d->hfield_data;
    const int nc = m->hf_ncol;
    for (int i = 1; i + 1 < m->hf_nrow; i++)
      for (int j = 1; j + 1 < nc; j++) {
        double mean = 0.25 * ((z[(i - 1) * nc + j] + z[(i + 1) * nc + j]) + (z[i * nc + j - 1] + z[i * nc + j + 1]));
        m->hf_convex[(size_t)i * nc + j] = z[i * nc + j] - mean > 1e-9 ? 1 : 0;
      }
  }
  auto moves = [&](int b) {
    for (; b > 0; b = m->body_parent[b]) if (m->body_jnt[b] >= 0) return true;
    return false;
  };
  int cmax = 0;
  for (int g1 = 0; g1 < m->ng; g1++)
    for (int g2 = g1 + 1; g2 < m->ng; g2++) {
      int b1 = m->geom_body[g1], b2 = m->geom_body[g2];
      if (b1 == b2) continue;
      if ((b1 > 0 && m->body_parent[b2] == b1) || (b2 > 0 && m->body_parent[b1] == b2)) continue;
      if (!((d->geom_contype[g1] & d->geom_conaffinity[g2]) || (d->geom_contype[g2] & d->geom_conaffinity[g1]))) continue;
      if (!moves(b1) && !moves(b2)) continue;
      int a = g1, b = g2;
      if (m->geom_type[b] < m->geom_type[a] || (m->geom_type[b] == m->geom_type[a] && b2 == 0 && b1 != 0))
        std::swap(a, b);
      if (m->geom_type[b] == B3P_GEOM_HFIELD) std::swap(a, b);   // the terrain is geom1
      int ta = m->geom_type[a], tb = m->geom_type[b], nmax = 0;
      if (ta == B3P_GEOM_HFIELD && tb == B3P_GEOM_SPHERE) nmax = 1;
      else if (ta == B3P_GEOM_HFIELD && tb == B3P_GEOM_CAPSULE) nmax = 2;
      else if (ta == B3P_GEOM_HFIELD && tb == B3P_GEOM_BOX) nmax = 4;
      else if (ta == B3P_GEOM_PLANE && tb == B3P_GEOM_SPHERE) nmax = 1;
      else if (ta == B3P_GEOM_PLANE && tb == B3P_GEOM_CAPSULE) nmax = 2;
      else if (ta == B3P_GEOM_PLANE && tb == B3P_GEOM_BOX) nmax = 4;
      else if (ta == B3P_GEOM_BOX && tb == B3P_GEOM_BOX) nmax = 8;
      else {
        delete m;
        return fail(B3P_ERR_UNSUPPORTED, "geom pair of types (%d, %d) is not supported", ta, tb);
      }
      if (ta == B3P_GEOM_PLANE && m->geom_body[a] != 0) return bad(B3P_ERR_UNSUPPORTED, "plane geoms must belong to the world body");
      int ba = m->geom_body[a], bb = m->geom_body[b];
      if (ba != 0 && bb != 0) {
        // two moving bodies: different kinematic trees couple through a dense Hessian
        if (m->body_root[ba] == m->body_root[bb])
          return bad(B3P_ERR_UNSUPPORTED, "contacts within one kinematic tree (self-collision) are not supported");
        m->dense = 1;
      }
      m->pair_g1.push_back(a);
      m->pair_g2.push_back(b);
      cmax += nmax;
    }
  m->npair = (int)m->pair_g1.size();
  m->ncon_max = std::min(cmax, d->contact_cap);
  if (m->dense && m->nv > 32) return bad(B3P_ERR_UNSUPPORTED, "cross-tree contacts need nv <= 32");
  for (int p = 0; p < m->npair; p++) {
    int l1 = 0, l2 = 0, b1 = m->geom_body[m->pair_g1[p]], b2 = m->geom_body[m->pair_g2[p]];
    if (b1 > 0 && m->body_dl[b1] >= 0) l1 = m->dof_rowlen[m->body_dl[b1]];
    if (b2 > 0 && m->body_dl[b2] >= 0) l2 = m->dof_rowlen[m->body_dl[b2]];
    if (l1 + l2 > 32) return bad(B3P_ERR_UNSUPPORTED, "a contact pair's two chains exceed 32 dofs");
  }
  for (int q = 0; q < 32; q++)
    for (int p = 0; p <= q; p++) m->tri_pq.push_back(p | q << 5);
  // options
  m->h = (float)d->timestep;
  for (int k = 0; k < 3; k++) m->grav[k] = (float)d->gravity[k];
  double tc = std::max(d->solref[0], 2 * d->timestep), zeta = d->solref[1], dmax = d->solimp[1];
  m->ref_b = (float)(2 / (dmax * tc));
  m->ref_k = (float)(1 / (dmax * dmax * tc * tc * zeta * zeta));
  for (int k = 0; k < 5; k++) m->imp[k] = (float)d->solimp[k];
  m->newton_iter = d->newton_iterations;
  m->ls_iter = d->ls_iterations;
  m->tol = (float)d->newton_tolerance;
  m->pivot_tau = (float)d->pivot_tau;
  m->push_period = d->push_period;
  m->push_sigma = (float)d->push_sigma;
  // per-world shared-memory layout (floats, each array 16-byte aligned)
  int off = 0;
  auto A = [&](int n) { int o = off; off += pad4(std::max(n, 1)); return o; };
  int nv = m->nv, nc = std::max(m->ncon_max, 1);
  m->o[O_QPOS] = A(m->nq); m->o[O_QVEL] = A(nv); m->o[O_QACC] = A(nv); m->o[O_QS] = A(nv); m->o[O_FRC] = A(nv);
  m->o[O_CTRL] = A(m->nu); m->o[O_KP] = A(m->nu); m->o[O_KD] = A(m->nu); m->o[O_MS] = A(nb);
  m->o[O_XPOS] = A(3 * nb); m->o[O_XQUAT] = A(4 * nb); m->o[O_XMAT] = A(9 * nb);
  m->o[O_CDOF] = A(6 * nv); m->o[O_CVEL] = A(6 * nb); m->o[O_UNION] = A(U_STRIDE * nb);
  // tree mode: H's factor has its own rows (the rows off the contacts' chains are M's
  // factor rows, refactored rows are rebuilt from M's factor every Newton iteration);
  // dense mode: the dense H overwrites the factor of M once the rows are done
  m->o[O_M] = A(m->nM); m->o[O_L] = A(m->dense ? std::max(m->nM, nv * nv) : m->nM);
  m->o[O_H] = m->dense ? m->o[O_L] : A(m->nM);
  m->o[O_HDIAG] = A(nv);
  m->o[O_MA] = A(nv); m->o[O_MP] = A(nv); m->o[O_G] = A(nv); m->o[O_P] = A(nv);
  // the per-dof CRBA temporary lives in the contact region, which is free until collision
  m->o[O_CON] = A(std::max(C_STRIDE * nc, 6 * nv)); m->o[O_TMP6] = m->o[O_CON];
  m->o[O_CONI] = A(CI_STRIDE * nc); m->o[O_MISC] = A(8);
  m->o[O_LIM] = A(LM_STRIDE * std::max((int)m->lim_dof.size(), 1));
  m->smem_floats = off;
  *out = m;
  return B3P_OK;
}

void b3p_model_destroy(b3p_model *m) { delete m; }

b3p_status b3p_model_info(const b3p_model *m, int32_t *out) {
  if (!m || !out) return fail(B3P_ERR_INVALID_ARG, "null argument");
  out[0] = m->nq; out[1] = m->nv; out[2] = m->nu; out[3] = m->nb; out[4] = m->ng; out[5] = m->npair;
  out[6] = m->ncon_max; out[7] = m->nM;
  return B3P_OK;
}

}  // extern "C"

namespace {

// byte layout of one batch inside the caller's buffer
struct Layout {
  uint64_t counter = 0, order = 0, solve_order = 0, solve_key = 0, lane_order = 0, solve_counts = 0, ws = ~0ull;
  uint64_t dbatch = 0, total = 0, model_bytes = 0, state_off = 0, state_bytes = 0, param_bytes = 0, contact_bytes = 0,
           scratch_bytes = 0;
  std::vector<uint64_t> model_off;                    // per distinct model index (== group here)
  struct G {
    uint64_t qpos, qvel, qacc, step, rng, seed, status, stats, hist, shist, fric, ms, kp, kd, inert, con, ncon,
        scratch;
  };
  std::vector<G> g;
};

// blob of one model: DModel header then the arrays; returns its size and fills offsets
struct Blob {
  std::vector<char> bytes;
  template <class T>
  uint64_t put(const std::vector<T> &v) {
    uint64_t off = align_up(bytes.size(), 16);
    bytes.resize(off + std::max<size_t>(v.size(), 1) * sizeof(T) + 16, 0);
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    bytes.resize(off + std::max<size_t>(v.size(), 1) * sizeof(T));
    return off;
  }
};

int model_maxchain(const b3p_model *m) {
  int mc = 1;
  for (int len : m->dof_rowlen) mc = std::max(mc, len);
  return mc;
}

// shared-memory bytes of a 32-world lane solve CTA for model m, or 0 when the model's
// solves cannot run one world per lane (dense Hessian, joint limits, no contacts, cdof
// larger than the factor area it is staged in)
int lane_solve_bytes(const b3p_model *m) {
  if (m->dense || !m->lim_dof.empty() || m->ncon_max <= 0 || 6 * m->nv > m->nM) return 0;
  LaneLayout o = lane_layout(m->nM, m->nv, model_maxchain(m));
  return o.total * B3P_LANE_STRIDE * 4;
}

uint64_t build_blob(const b3p_model *m, char *dev_base, Blob &blob) {
  blob.bytes.assign(align_up(sizeof(DModel), 16), 0);
  DModel dm{};
  auto P = [&](auto &dst, const auto &vec) {
    uint64_t off = blob.put(vec);
    dst = reinterpret_cast<std::remove_reference_t<decltype(dst)>>(dev_base ? dev_base + off : nullptr);
  };
  dm.nb = m->nb; dm.nj = m->nj; dm.nu = m->nu; dm.ng = m->ng; dm.nq = m->nq; dm.nv = m->nv; dm.npair = m->npair;
  dm.ncon_max = m->ncon_max; dm.nM = m->nM; dm.maxlevel = m->maxlevel;
  dm.nq_pad = pad4(m->nq); dm.nv_pad = pad4(m->nv); dm.nu_pad = pad4(std::max(m->nu, 1)); dm.nb_pad = pad4(m->nb);
  dm.first_free_dof = m->first_free_dof;
  dm.newton_iter = m->newton_iter; dm.ls_iter = m->ls_iter; dm.push_period = m->push_period;
  dm.h = m->h; for (int k = 0; k < 3; k++) dm.grav[k] = m->grav[k];
  dm.ref_b = m->ref_b; dm.ref_k = m->ref_k; for (int k = 0; k < 5; k++) dm.imp[k] = m->imp[k];
  dm.tol = m->tol; dm.pivot_tau = m->pivot_tau; dm.push_sigma = m->push_sigma;
  dm.smem_floats = m->smem_floats;
  dm.dense = m->dense;
  dm.maxchain = model_maxchain(m);
  dm.scratch_doubles = B3P_SCRATCH_DOUBLES(m->nM, m->nv, m->dense);
  int *o = &dm.o_qpos;
  for (int k = 0; k < 28; k++) o[k] = m->o[k];
  dm.nlim = (int)m->lim_dof.size(); dm.dcmotor = m->dcmotor; dm.act_delay = m->act_delay;
  P(dm.lim_dof, m->lim_dof); P(dm.lim_qadr, m->lim_qadr); P(dm.lim_range, m->lim_range); P(dm.act_dcm, m->act_dcm);
  dm.hf_nrow = m->hf_nrow; dm.hf_ncol = m->hf_ncol; dm.hf_hx = m->hf_hx; dm.hf_hy = m->hf_hy;
  P(dm.hf_data, m->hf_data);
  P(dm.hf_convex, m->hf_convex);
  P(dm.body_parent, m->body_parent); P(dm.body_jnt, m->body_jnt); P(dm.body_root, m->body_root);
  P(dm.body_dl, m->body_dl); P(dm.level_body, m->level_body); P(dm.level_start, m->level_start);
  P(dm.child_start, m->child_start); P(dm.child_list, m->child_list);
  P(dm.body_geom_adr, m->body_geom_adr); P(dm.body_geom, m->body_geom);
  P(dm.body_pos, m->body_pos); P(dm.body_quat, m->body_quat); P(dm.body_mass, m->body_mass);
  P(dm.body_ipos, m->body_ipos); P(dm.body_inertia, m->body_inertia);
  P(dm.jnt_type, m->jnt_type); P(dm.jnt_qadr, m->jnt_qadr); P(dm.jnt_dadr, m->jnt_dadr);
  P(dm.jnt_axis, m->jnt_axis); P(dm.jnt_pos, m->jnt_pos); P(dm.jnt_noise, m->jnt_noise); P(dm.qpos_reset, m->qpos_reset);
  P(dm.dof_body, m->dof_body); P(dm.dof_jnt, m->dof_jnt); P(dm.dof_rowadr, m->dof_rowadr); P(dm.dof_rowlen, m->dof_rowlen);
  P(dm.colind, m->colind); P(dm.entry_row, m->entry_row); P(dm.col_start, m->col_start); P(dm.col_k, m->col_k);
  P(dm.col_pos, m->col_pos); P(dm.dof_armature, m->dof_armature);
  P(dm.act_qadr, m->act_qadr); P(dm.act_dadr, m->act_dadr); P(dm.act_kp, m->act_kp); P(dm.act_kd, m->act_kd);
  P(dm.geom_type, m->geom_type); P(dm.geom_body, m->geom_body); P(dm.geom_size, m->geom_size);
  P(dm.geom_pos, m->geom_pos); P(dm.geom_mat, m->geom_mat); P(dm.geom_friction, m->geom_friction);
  P(dm.pair_g1, m->pair_g1); P(dm.pair_g2, m->pair_g2);
  P(dm.ltdl_adr, m->ltdl_adr); P(dm.chain_adr, m->chain_adr); P(dm.ltdl_ops, m->ltdl_ops);
  P(dm.chain_ops, m->chain_ops); P(dm.body_mask, m->body_mask); P(dm.tri_pq, m->tri_pq);
  P(dm.dof_mask, m->dof_mask); P(dm.level_rec, m->level_rec);
  P(dm.sym_start, m->sym_start); P(dm.sym_ops, m->sym_ops); P(dm.entry_ops, m->entry_ops);
  std::memcpy(blob.bytes.data(), &dm, sizeof dm);
  return align_up(blob.bytes.size(), 256);
}

b3p_status make_layout(const b3p_model *const *models, const int32_t *nworld, int32_t nmodels, const b3p_options &opt,
                       Layout &L) {
  if (!models || !nworld || nmodels < 1) return fail(B3P_ERR_INVALID_ARG, "need at least one model group");
  if (nmodels > B3P_MAXGROUP) return fail(B3P_ERR_UNSUPPORTED, "at most %d model groups per batch", B3P_MAXGROUP);
  if (opt.history < 0 || opt.history > 64) return fail(B3P_ERR_INVALID_ARG, "history outside 0..64");
  if (opt.working_set < 0 || opt.working_set > 3) return fail(B3P_ERR_INVALID_ARG, "working_set outside 0..3");
  if (opt.schedule < 0 || opt.schedule > 1) return fail(B3P_ERR_INVALID_ARG, "schedule outside 0..1");
  if (opt.lane_solve < 0 || opt.lane_solve > 1) return fail(B3P_ERR_INVALID_ARG, "lane_solve outside 0..1");
  if (opt.smem_scratch < 0 || opt.smem_scratch > 1) return fail(B3P_ERR_INVALID_ARG, "smem_scratch outside 0..1");
  if (opt.lane_solve == 1 && (opt.working_set < 2 || opt.schedule != 1))
    return fail(B3P_ERR_INVALID_ARG, "lane_solve needs a staged placement (working_set 2 or 3) with schedule 1");
  uint64_t off = 0;
  auto A = [&](uint64_t n) { uint64_t o = off; off = align_up(off + std::max<uint64_t>(n, 1), 256); return o; };
  L.dbatch = A(sizeof(DBatch));
  int total = 0;
  for (int g = 0; g < nmodels; g++) total += std::max(nworld[g], 0);
  L.counter = A(4);
  L.order = A(4 * (uint64_t)total);
  L.solve_order = A(4 * (uint64_t)total);
  L.solve_key = A((uint64_t)total);
  L.lane_order = A(4 * ((uint64_t)total + 32ull * nmodels));
  L.solve_counts = A(8);
  uint64_t m0 = off;
  for (int g = 0; g < nmodels; g++) {
    if (!models[g]) return fail(B3P_ERR_INVALID_ARG, "null model in group %d", g);
    if (nworld[g] < 0) return fail(B3P_ERR_INVALID_ARG, "negative world count in group %d", g);
    Blob blob;
    L.model_off.push_back(A(build_blob(models[g], nullptr, blob)));
  }
  L.model_bytes = off - m0;
  // state region (contiguous, for save/restore)
  L.state_off = off;
  L.g.resize(nmodels);
  for (int g = 0; g < nmodels; g++) {
    const b3p_model *m = models[g];
    uint64_t W = (uint64_t)nworld[g];
    auto &G = L.g[g];
    G.qpos = A(4 * W * pad4(m->nq)); G.qvel = A(4 * W * pad4(m->nv)); G.qacc = A(4 * W * pad4(m->nv));
    G.step = A(4 * W); G.rng = A(4 * W); G.seed = A(8 * W); G.status = A(4 * W); G.stats = A(16 * W);
    G.hist = m->act_delay > 0 ? A(4 * W * (uint64_t)m->act_delay * pad4(std::max(m->nu, 1))) : ~0ull;
    G.shist = opt.history > 0 ? A(4 * W * (uint64_t)opt.history * (m->nq + m->nv)) : ~0ull;
  }
  L.state_bytes = off - L.state_off;
  uint64_t p0 = off;
  for (int g = 0; g < nmodels; g++) {
    const b3p_model *m = models[g];
    uint64_t W = (uint64_t)nworld[g];
    auto &G = L.g[g];
    G.fric = A(4 * W); G.ms = A(4 * W * pad4(m->nb)); G.kp = A(4 * W * pad4(std::max(m->nu, 1)));
    G.inert = A(40 * W * m->nb);
    G.kd = A(4 * W * pad4(std::max(m->nu, 1)));
  }
  L.param_bytes = off - p0;
  uint64_t c0 = off;
  for (int g = 0; g < nmodels; g++) {
    const b3p_model *m = models[g];
    uint64_t W = (uint64_t)nworld[g];
    auto &G = L.g[g];
    if (opt.write_contacts) {
      G.con = A(4 * W * std::max(m->ncon_max, 1) * 24);
      G.ncon = A(4 * W);
    } else {
      G.con = G.ncon = ~0ull;
    }
  }
  L.contact_bytes = off - c0;
  uint64_t s0 = off;
  for (int g = 0; g < nmodels; g++) {
    const b3p_model *m = models[g];
    L.g[g].scratch = A(8 * (uint64_t)nworld[g] * B3P_SCRATCH_DOUBLES(m->nM, m->nv, m->dense));
  }
  L.scratch_bytes = off - s0;
  L.ws = ~0ull;
  if (opt.working_set >= 1 && opt.working_set <= 3) {
    uint64_t n = 0;
    for (int g = 0; g < nmodels; g++) n += (uint64_t)nworld[g] * models[g]->smem_floats * 4;
    L.ws = A(n);
  }
  L.total = off;
  return B3P_OK;
}

b3p_options defaults(const b3p_options *opt) {
  b3p_options o{};
  if (opt) o = *opt;
  return o;
}

int has_limits(const b3p_batch *b) {
  for (auto *m : b->models)
    if (!m->lim_dof.empty()) return 1;
  return 0;
}

b3p_status configure_launch(b3p_batch *b) {
  int dev = 0, nsm = 0, smem_optin = 0;
  CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem limit");
  int wpb = b->opt.warps_per_block > 0 ? b->opt.warps_per_block : 4;
  wpb = std::min(wpb, 8);
  while (wpb > 1 && (uint64_t)wpb * b->smem_floats * 4 > (uint64_t)smem_optin) wpb--;
  if ((uint64_t)wpb * b->smem_floats * 4 > (uint64_t)smem_optin)
    return fail(B3P_ERR_UNSUPPORTED, "one world needs %d bytes of shared memory (limit %d)", b->smem_floats * 4, smem_optin);
  b->wpb = wpb;
  b->smem_bytes = b->opt.working_set != 0 ? 0 : wpb * b->smem_floats * 4;
  int per_sm = 0;
  int rc = b3p_step_occupancy(b->smem_bytes, wpb, &per_sm);
  if (rc != 0) return cuda_fail((cudaError_t)rc, "occupancy query");
  per_sm = std::max(per_sm, 1);
  if (b->opt.blocks_per_sm > 0) per_sm = std::min(per_sm, b->opt.blocks_per_sm);
  int need = (b->total_world + wpb - 1) / wpb;
  b->grid = std::max(1, std::min(need, nsm * per_sm));
  b->aux_smem = 0;
  if (b->opt.working_set == 3 && B3P_SMOOTH_AUX && b->opt.smem_scratch == 0) {
    int bytes = std::min(wpb, 4) * b->host.aux_floats * 4;
    if (bytes > 0 && bytes <= smem_optin) {
      int rc2 = b3p_aux_prepare(bytes);
      if (rc2) return cuda_fail((cudaError_t)rc2, "smooth-launch scratch shared-memory limit");
      b->aux_smem = bytes;
    }
  }
  b->solve_smem = 0;
  if (b->opt.working_set >= 2 && B3P_SOLVE_AUX && b->opt.smem_scratch == 0) {
    int bytes = std::min(wpb, 4) * b->host.solve_aux_floats * 4;
    if (bytes > 0 && bytes <= smem_optin) {
      int rc2 = b3p_solve_aux_prepare(bytes);
      if (rc2) return cuda_fail((cudaError_t)rc2, "solve-launch scratch shared-memory limit");
      b->solve_smem = bytes;
    }
  }
  if (b->aux_smem || b->solve_smem) {   // keep only the blocks that cost no residency
    int smooth_ok = 0, solve_ok = 0;
    int rc2 = b3p_aux_fits(b->aux_smem, b->solve_smem, std::min(wpb, 4), &smooth_ok, &solve_ok);
    if (rc2) return cuda_fail((cudaError_t)rc2, "occupancy query");
    if (!smooth_ok) b->aux_smem = 0;
    if (!solve_ok) b->solve_smem = 0;
  }
  return B3P_OK;
}

}  // namespace

extern "C" {

b3p_status b3p_batch_plan(const b3p_model *const *models, const int32_t *nworld, int32_t nmodels,
                          const b3p_options *opt, b3p_sizes *out) {
  if (!out) return fail(B3P_ERR_INVALID_ARG, "null output");
  Layout L;
  b3p_status s = make_layout(models, nworld, nmodels, defaults(opt), L);
  if (s) return s;
  out->total_bytes = L.total;
  out->model_bytes = L.model_bytes;
  out->state_bytes = L.state_bytes;
  out->param_bytes = L.param_bytes;
  out->contact_bytes = L.contact_bytes;
  out->scratch_bytes = L.scratch_bytes;
  int tw = 0, sm = 0;
  for (int g = 0; g < nmodels; g++) { tw += nworld[g]; sm = std::max(sm, models[g]->smem_floats); }
  out->nworld = tw;
  out->smem_bytes_per_world = sm * 4;
  return B3P_OK;
}

b3p_status b3p_batch_create(const b3p_model *const *models, const int32_t *nworld, int32_t nmodels,
                            const b3p_options *opt, const b3p_buffers *bufs, void *stream, b3p_batch **out) {
  if (!out || !bufs) return fail(B3P_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  b3p_options o = defaults(opt);
  Layout L;
  b3p_status s = make_layout(models, nworld, nmodels, o, L);
  if (s) return s;
  if (!bufs->base || ((uintptr_t)bufs->base & 255)) return fail(B3P_ERR_INVALID_ARG, "buffer must be 256-byte aligned");
  if (bufs->bytes < L.total)
    return fail(B3P_ERR_WORKSPACE_TOO_SMALL, "buffer holds %llu bytes, batch needs %llu",
                (unsigned long long)bufs->bytes, (unsigned long long)L.total);
  cudaStream_t st = (cudaStream_t)stream;
  b3p_batch *b = new b3p_batch();
  b->opt = o;
  b->base = (char *)bufs->base;
  b->bytes = bufs->bytes;
  b->dev = (DBatch *)(b->base + L.dbatch);
  b->state_off = L.state_off;
  b->state_bytes = L.state_bytes;
  std::vector<Blob> blobs(nmodels);
  std::vector<std::vector<float>> params;
  int tw = 0, sm = 0;
  DBatch &H = b->host;
  std::memset(&H, 0, sizeof H);
  H.ngroup = nmodels;
  for (int g = 0; g < nmodels; g++) {
    const b3p_model *m = models[g];
    b->models.push_back(m);
    b->nworld.push_back(nworld[g]);
    b->world_start.push_back(tw);
    char *mb = b->base + L.model_off[g];
    build_blob(m, mb, blobs[g]);
    DGroup &G = H.g[g];
    auto &lg = L.g[g];
    G.m = (const DModel *)mb;
    G.world_start = tw;
    G.nworld = nworld[g];
    G.ctrl_offset = 0;
    for (int k = 0; k < g; k++) G.ctrl_offset += nworld[k] * models[k]->nu;
    G.qpos = (float *)(b->base + lg.qpos); G.qvel = (float *)(b->base + lg.qvel); G.qacc = (float *)(b->base + lg.qacc);
    G.step_count = (int *)(b->base + lg.step); G.rng_id = (int *)(b->base + lg.rng);
    G.seed = (uint32_t *)(b->base + lg.seed); G.status = (uint32_t *)(b->base + lg.status);
    G.stats = (int *)(b->base + lg.stats);
    G.friction = (float *)(b->base + lg.fric); G.mass_scale = (float *)(b->base + lg.ms);
    G.kp = (float *)(b->base + lg.kp); G.kd = (float *)(b->base + lg.kd);
    G.inertia = (float *)(b->base + lg.inert);
    G.con = o.write_contacts ? (float *)(b->base + lg.con) : nullptr;
    G.ncon = o.write_contacts ? (int *)(b->base + lg.ncon) : nullptr;
    G.scratch64 = (double *)(b->base + lg.scratch);
    G.ctrl_hist = lg.hist != ~0ull ? (float *)(b->base + lg.hist) : nullptr;
    G.state_hist = lg.shist != ~0ull ? (float *)(b->base + lg.shist) : nullptr;
    G.history = o.history > 0 ? o.history : 0;
    tw += nworld[g];
    sm = std::max(sm, m->smem_floats);
  }
  H.nworld = tw;
  H.smem_floats = sm;
  for (int g = 0; g < nmodels; g++) {
    const b3p_model *mg = models[g];
    H.aux_floats = std::max(H.aux_floats, pad4(AUX_CI * mg->nb + aux_region_floats(mg->nb, mg->nv)));
    H.solve_aux_floats = std::max(H.solve_aux_floats, pad4(mg->dense ? mg->nv * mg->nv : mg->nM) + 5 * pad4(mg->nv) +
                                                          (B3P_SOLVE_STAGE_INPUTS ? 2 * pad4(mg->nM) + pad4(6 * mg->nv) : 0));
  }
  H.schedule = o.schedule == 1 ? 1 : 0;
  H.ws = (o.working_set >= 1 && o.working_set <= 3) ? (float *)(b->base + L.ws) : nullptr;
  {
    long long acc = 0;   // per-group offsets (floats, multiples of 4) of the working-set region
    for (int g = 0; g < nmodels; g++) {
      H.g[g].ws_off4 = (int)(acc / 4);
      acc += (long long)nworld[g] * models[g]->smem_floats;
    }
    H.ws_floats = acc;
  }
  {
    // the lane solve: groups whose per-CTA block fits the device's shared memory
    int dev = 0, optin = 0, bytes = 0;
    if (o.lane_solve == 1) {
      cudaError_t ee = cudaGetDevice(&dev);
      if (ee == cudaSuccess) ee = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (ee) { delete b; return cuda_fail(ee, "shared-memory limit"); }
      for (int g = 0; g < nmodels; g++) {
        int need = lane_solve_bytes(models[g]);
        H.g[g].lane_ok = need > 0 && need <= optin;
        if (H.g[g].lane_ok) bytes = std::max(bytes, need);
      }
    }
    H.lane_solve = bytes > 0;
    H.lane_order = (int *)(b->base + L.lane_order);
    H.solve_counts = (int *)(b->base + L.solve_counts);
    b->lane_smem = bytes;
    if (bytes > 0) {
      int rc = b3p_lane_solve_prepare(bytes);
      if (rc) { delete b; return cuda_fail((cudaError_t)rc, "lane solve shared-memory limit"); }
    }
  }
  H.counter = (int *)(b->base + L.counter);
  H.order = (const int *)(b->base + L.order);
  H.solve_order = (int *)(b->base + L.solve_order);
  H.solve_key = (unsigned char *)(b->base + L.solve_key);
  b->counter = H.counter;
  // queue order: groups by decreasing per-world cost (nv^2 + contact slots), world order within
  std::vector<int> gorder(nmodels);
  for (int g = 0; g < nmodels; g++) gorder[g] = g;
  std::stable_sort(gorder.begin(), gorder.end(), [&](int x, int y) {
    auto cost = [&](int g) { return (long)models[g]->nv * models[g]->nv + 8L * models[g]->ncon_max; };
    return cost(x) > cost(y);
  });
  std::vector<int> order;
  for (int g : gorder)
    for (int w = 0; w < nworld[g]; w++) order.push_back(b->world_start[g] + w);
  b->total_world = tw;
  b->smem_floats = sm;
  auto cleanup = [&](b3p_status code) { delete b; return code; };
  cudaError_t e;
  for (int g = 0; g < nmodels; g++) {
    e = cudaMemcpyAsync(b->base + L.model_off[g], blobs[g].bytes.data(), blobs[g].bytes.size(), cudaMemcpyHostToDevice, st);
    if (e) return cleanup(cuda_fail(e, "model upload"));
  }
  e = cudaMemcpyAsync(b->dev, &H, sizeof H, cudaMemcpyHostToDevice, st);
  if (e) return cleanup(cuda_fail(e, "batch upload"));
  if (!order.empty()) {
    e = cudaMemcpyAsync(b->base + L.order, order.data(), 4 * order.size(), cudaMemcpyHostToDevice, st);
    if (e) return cleanup(cuda_fail(e, "order upload"));
  }
  e = cudaMemsetAsync(b->base + L.state_off, 0, L.state_bytes, st);
  if (e) return cleanup(cuda_fail(e, "state clear"));
  e = cudaMemsetAsync(b->base + L.solve_key, 64, (size_t)std::max(tw, 1), st);   // bucket 64: idle
  if (e) return cleanup(cuda_fail(e, "solve key clear"));
  // default per-world parameters
  for (int g = 0; g < nmodels; g++) {
    const b3p_model *m = models[g];
    const DGroup &G = H.g[g];
    size_t W = nworld[g];
    int nbp = pad4(m->nb), nup = pad4(std::max(m->nu, 1));
    params.emplace_back(W, 1.f);
    e = cudaMemcpyAsync(G.friction, params.back().data(), 4 * W, cudaMemcpyHostToDevice, st);
    if (e) return cleanup(cuda_fail(e, "param upload"));
    params.emplace_back(W * nbp, 1.f);
    e = cudaMemcpyAsync(G.mass_scale, params.back().data(), 4 * W * nbp, cudaMemcpyHostToDevice, st);
    if (e) return cleanup(cuda_fail(e, "param upload"));
    std::vector<float> kp(W * nup, 0.f), kd(W * nup, 0.f);
    for (size_t w = 0; w < W; w++)
      for (int u = 0; u < m->nu; u++) { kp[w * nup + u] = m->act_kp[u]; kd[w * nup + u] = m->act_kd[u]; }
    params.push_back(std::move(kp));
    e = cudaMemcpyAsync(G.kp, params.back().data(), 4 * W * nup, cudaMemcpyHostToDevice, st);
    if (e) return cleanup(cuda_fail(e, "param upload"));
    params.push_back(std::move(kd));
    e = cudaMemcpyAsync(G.kd, params.back().data(), 4 * W * nup, cudaMemcpyHostToDevice, st);
    if (e) return cleanup(cuda_fail(e, "param upload"));
    std::vector<float> bi(W * 10 * m->nb);
    for (size_t w = 0; w < W; w++)
      for (int bb = 0; bb < m->nb; bb++) {
        float *o = &bi[(w * m->nb + bb) * 10];
        o[0] = m->body_mass[bb];
        for (int k = 0; k < 3; k++) o[1 + k] = m->body_ipos[3 * bb + k];
        for (int k = 0; k < 6; k++) o[4 + k] = m->body_inertia[6 * bb + k];
      }
    params.push_back(std::move(bi));
    e = cudaMemcpyAsync(G.inertia, params.back().data(), 40 * W * m->nb, cudaMemcpyHostToDevice, st);
    if (e) return cleanup(cuda_fail(e, "param upload"));
  }
  if (o.write_contacts) {
    uint64_t c0 = L.g[0].con;
    e = cudaMemsetAsync(b->base + c0, 0, L.contact_bytes, st);
    if (e) return cleanup(cuda_fail(e, "contact clear"));
  }
  e = cudaStreamSynchronize(st);
  if (e) return cleanup(cuda_fail(e, "batch create"));
  b3p_status cs = configure_launch(b);
  if (cs) return cleanup(cs);
  *out = b;
  return B3P_OK;
}

void b3p_batch_destroy(b3p_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

b3p_status b3p_batch_info(const b3p_batch *b, int32_t *out, int32_t cap) {
  if (!b || !out) return fail(B3P_ERR_INVALID_ARG, "null argument");
  int ng = (int)b->models.size();
  std::vector<int32_t> v = {b->total_world, ng, 0, 0};
  for (int g = 0; g < ng; g++) {
    v[2] += b->nworld[g] * b->models[g]->nq;
    v[3] += b->nworld[g] * b->models[g]->nv;
  }
  for (int g = 0; g < ng; g++) { v.push_back(b->world_start[g]); v.push_back(b->nworld[g]); }
  if (cap < (int)v.size()) return fail(B3P_ERR_INVALID_ARG, "info needs %d entries", (int)v.size());
  std::copy(v.begin(), v.end(), out);
  return B3P_OK;
}

b3p_status b3p_batch_launch_info(const b3p_batch *b, int32_t *out, int32_t cap) {
  if (!b || !out) return fail(B3P_ERR_INVALID_ARG, "null argument");
  if (cap < 5) return fail(B3P_ERR_INVALID_ARG, "launch info needs 5 entries");
  out[0] = b->wpb; out[1] = b->grid; out[2] = b->aux_smem; out[3] = b->solve_smem; out[4] = b->lane_smem;
  return B3P_OK;
}

b3p_status b3p_reset(b3p_batch *b, uint64_t seed, const int32_t *world_ids, const int32_t *rng_ids, int32_t n,
                     void *stream) {
  if (!b) return fail(B3P_ERR_INVALID_ARG, "null batch");
  if (!world_ids) n = b->total_world;
  if (n < 0) return fail(B3P_ERR_INVALID_ARG, "negative count");
  int rc = b3p_launch_reset(b->dev, b->total_world, (uint32_t)seed, (uint32_t)(seed >> 32), world_ids, rng_ids, n, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "reset launch");
  return B3P_OK;
}

b3p_status b3p_set_world_param(b3p_batch *b, int32_t group, b3p_param field, const float *src, void *stream) {
  if (!b || !src) return fail(B3P_ERR_INVALID_ARG, "null argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  const b3p_model *m = b->models[group];
  DGroup &G = b->host.g[group];
  size_t W = b->nworld[group];
  if (W == 0) return B3P_OK;
  float *dst;
  int n, npad;
  switch (field) {
    case B3P_PARAM_FRICTION_SCALE: dst = G.friction; n = 1; npad = 1; break;
    case B3P_PARAM_MASS_SCALE: dst = G.mass_scale; n = m->nb; npad = pad4(m->nb); break;
    case B3P_PARAM_KP: dst = G.kp; n = m->nu; npad = pad4(std::max(m->nu, 1)); break;
    case B3P_PARAM_KD: dst = G.kd; n = m->nu; npad = pad4(std::max(m->nu, 1)); break;
    case B3P_PARAM_BODY_INERTIA: dst = G.inertia; n = 10 * m->nb; npad = 10 * m->nb; break;
    default: return fail(B3P_ERR_INVALID_ARG, "unknown parameter");
  }
  if (n == 0) return B3P_OK;
  CUDA_TRY(cudaMemcpy2DAsync(dst, 4 * npad, src, 4 * n, 4 * n, W, cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
           "param copy");
  if (field == B3P_PARAM_BODY_INERTIA && !G.inertia_custom) {
    // from now on the kernels read the per-world inertias (the flag's host copy lives as
    // long as the batch, as the asynchronous copy needs)
    G.inertia_custom = 1;
    CUDA_TRY(cudaMemcpyAsync(&b->dev->g[group].inertia_custom, &G.inertia_custom, sizeof(int), cudaMemcpyHostToDevice,
                             (cudaStream_t)stream),
             "inertia flag");
  }
  return B3P_OK;
}

b3p_status b3p_step_profile(b3p_batch *b, const float *ctrl, int32_t decimation, float *stage_ms,
                            int32_t *launches, void *stream) {
  if (!b || !stage_ms) return fail(B3P_ERR_INVALID_ARG, "null batch or stage_ms");
  if (decimation < 1) return fail(B3P_ERR_INVALID_ARG, "decimation must be >= 1");
  if (b->opt.working_set < 2) return fail(B3P_ERR_UNSUPPORTED, "per-stage timing needs a staged placement");
  bool need_ctrl = false;
  for (auto *m : b->models) need_ctrl |= m->nu > 0;
  if (need_ctrl && !ctrl) return fail(B3P_ERR_INVALID_ARG, "ctrl is required: a group has actuators");
  if (b->total_world == 0) return B3P_OK;
  int nev = 3 + 6 * decimation;
  std::vector<cudaEvent_t> ev(nev, nullptr);
  b3p_status out = B3P_OK;
  for (int i = 0; i < nev && out == B3P_OK; i++)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) out = fail(B3P_ERR_CUDA, "cudaEventCreate");
  if (out == B3P_OK) {
    int rc = b3p_launch_staged_events(b->dev, b->total_world, ctrl, decimation, std::min(b->wpb, 4), has_limits(b),
                                      b->opt.schedule == 1, b->lane_smem, b->solve_smem, b->models.size() == 1,
                                      stream, reinterpret_cast<void *const *>(ev.data()));
    if (rc) out = cuda_fail((cudaError_t)rc, "staged step launch");
    else if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) out = fail(B3P_ERR_CUDA, "stream sync");
  }
  if (out == B3P_OK) {
    // launch k runs between events k and k + 1: stage of launch k
    for (int k = 0; k + 1 < nev; k++) {
      int stage = k == 0 ? 0 : (k == nev - 2 ? B3P_NSTAGES - 1 : 1 + (k - 1) % 6);
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) { out = fail(B3P_ERR_CUDA, "event time"); break; }
      stage_ms[stage] += ms;
      if (launches) launches[stage] += 1;
    }
  }
  for (auto e : ev)
    if (e) cudaEventDestroy(e);
  return out;
}

b3p_status b3p_fp32_peak(int32_t reps, double *flops_per_s_host, int32_t *sm_count_host, void *stream) {
  if (!flops_per_s_host || !sm_count_host) return fail(B3P_ERR_INVALID_ARG, "null output");
  if (reps < 1) return fail(B3P_ERR_INVALID_ARG, "reps must be >= 1");
  int sms = 0;
  int rc = b3p_fma_probe(reps, flops_per_s_host, &sms, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "FMA probe");
  *sm_count_host = sms;
  return B3P_OK;
}

b3p_status b3p_step(b3p_batch *b, const float *ctrl, int32_t decimation, void *stream) {
  if (!b) return fail(B3P_ERR_INVALID_ARG, "null batch");
  if (decimation < 1) return fail(B3P_ERR_INVALID_ARG, "decimation must be >= 1");
  bool need_ctrl = false;
  for (auto *m : b->models) need_ctrl |= m->nu > 0;
  if (need_ctrl && !ctrl) return fail(B3P_ERR_INVALID_ARG, "ctrl is required: a group has actuators");
  if (b->total_world == 0) return B3P_OK;
  if (b->opt.working_set >= 2) {
    int rc = b3p_launch_staged(b->dev, b->total_world, ctrl, decimation, std::min(b->wpb, 4), has_limits(b),
                               b->opt.schedule == 1, b->opt.working_set == 3, b->lane_smem, b->aux_smem,
                               b->solve_smem, b->models.size() == 1, stream);
    if (rc) return cuda_fail((cudaError_t)rc, "staged step launch");
    return B3P_OK;
  }
  if (b->opt.schedule == 1)
    CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int), (cudaStream_t)stream), "queue reset");
  int rc = b3p_launch_step(b->dev, b->total_world, ctrl, decimation, b->wpb, b->grid, b->smem_bytes, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "step launch");
  return B3P_OK;
}

b3p_status b3p_step_static_scratch(b3p_batch *b, const float *ctrl, int32_t decimation, void *stream) {
  if (!b) return fail(B3P_ERR_INVALID_ARG, "null batch");
  if (decimation < 1) return fail(B3P_ERR_INVALID_ARG, "decimation must be >= 1");
  bool need_ctrl = false;
  uint64_t need = 0;
  for (size_t g = 0; g < b->models.size(); g++) {
    need_ctrl |= b->models[g]->nu > 0;
    need += (uint64_t)b->nworld[g] * (uint64_t)B3P_SCRATCH_DOUBLES(b->models[g]->nM, b->models[g]->nv, b->models[g]->dense);
  }
  if (need_ctrl && !ctrl) return fail(B3P_ERR_INVALID_ARG, "ctrl is required: a group has actuators");
  if (b->opt.working_set != 0)
    return fail(B3P_ERR_UNSUPPORTED, "this entry point keeps working sets in shared memory: create the batch "
                                     "with working_set = 0");
  if (need > (uint64_t)B3P_STATIC_SCRATCH_DOUBLES)
    return fail(B3P_ERR_INVALID_ARG,
                "batch needs %llu doubles of FP64 workspace, the library's fixed array holds %llu; "
                "step it with b3p_step",
                (unsigned long long)need, (unsigned long long)B3P_STATIC_SCRATCH_DOUBLES);
  if (b->total_world == 0) return B3P_OK;
  // the static kernel walks worlds in index order (no queue), so the schedule option
  // and the queue counter play no part here
  int rc = b3p_launch_step_static(b->dev, b->total_world, ctrl, decimation, b->wpb, b->smem_bytes, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "static-scratch step launch");
  return B3P_OK;
}

b3p_status b3p_step_capture(b3p_batch *b, const float *ctrl_base, int64_t stride, int32_t decimation, int32_t nsteps,
                            void *stream) {
  if (!b || nsteps < 1 || decimation < 1) return fail(B3P_ERR_INVALID_ARG, "bad capture arguments");
  if (!stream) return fail(B3P_ERR_INVALID_ARG, "capture needs a non-default stream");
  cudaStream_t st = (cudaStream_t)stream;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
  b3p_status s = B3P_OK;
  for (int i = 0; i < nsteps && s == B3P_OK; i++) s = b3p_step(b, ctrl_base ? ctrl_base + (int64_t)i * stride : nullptr, decimation, stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s) { if (g) cudaGraphDestroy(g); return s; }
  if (e) return cuda_fail(e, "end capture");
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e) { cudaGraphDestroy(g); b->graph = nullptr; return cuda_fail(e, "graph instantiate"); }
  b->graph_version = b->layout_version;
  return B3P_OK;
}

b3p_status b3p_graph_launch(b3p_batch *b, void *stream) {
  if (!b || !b->exec) return fail(B3P_ERR_INVALID_ARG, "no captured graph");
  if (b->graph_version != b->layout_version) return fail(B3P_ERR_GRAPH_STALE, "batch layout changed since capture");
  CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "graph launch");
  return B3P_OK;
}

}  // extern "C"

namespace {
// per-group (pointer, row stride, row width, element size) of a state field
bool field_view(const b3p_batch *b, int g, b3p_field f, char **ptr, size_t *pitch, size_t *width) {
  const b3p_model *m = b->models[g];
  const DGroup &G = b->host.g[g];
  switch (f) {
    case B3P_FIELD_QPOS: *ptr = (char *)G.qpos; *pitch = 4 * pad4(m->nq); *width = 4 * m->nq; return true;
    case B3P_FIELD_QVEL: *ptr = (char *)G.qvel; *pitch = 4 * pad4(m->nv); *width = 4 * m->nv; return true;
    case B3P_FIELD_QACC: *ptr = (char *)G.qacc; *pitch = 4 * pad4(m->nv); *width = 4 * m->nv; return true;
    case B3P_FIELD_STATUS: *ptr = (char *)G.status; *pitch = 4; *width = 4; return true;
    case B3P_FIELD_STATS: *ptr = (char *)G.stats; *pitch = 16; *width = 16; return true;
    case B3P_FIELD_STEP_COUNT: *ptr = (char *)G.step_count; *pitch = 4; *width = 4; return true;
  }
  return false;
}

b3p_status copy_field(b3p_batch *b, b3p_field f, char *dense, size_t bytes, bool to_state, void *stream) {
  if (!b || (!dense && bytes > 0)) return fail(B3P_ERR_INVALID_ARG, "null argument");
  size_t need = 0;
  for (int g = 0; g < (int)b->models.size(); g++) {
    char *p; size_t pitch, width;
    if (!field_view(b, g, f, &p, &pitch, &width)) return fail(B3P_ERR_INVALID_ARG, "unknown field");
    need += width * b->nworld[g];
  }
  if (bytes != need) return fail(B3P_ERR_INVALID_ARG, "field needs %zu bytes, got %zu", need, bytes);
  if (need == 0) return B3P_OK;   // no worlds: nothing to copy (a null buffer is fine)
  size_t off = 0;
  for (int g = 0; g < (int)b->models.size(); g++) {
    char *p; size_t pitch, width;
    field_view(b, g, f, &p, &pitch, &width);
    size_t W = b->nworld[g];
    if (W == 0 || width == 0) continue;
    cudaError_t e = to_state
        ? cudaMemcpy2DAsync(p, pitch, dense + off, width, width, W, cudaMemcpyDeviceToDevice, (cudaStream_t)stream)
        : cudaMemcpy2DAsync(dense + off, width, p, pitch, width, W, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e) return cuda_fail(e, "state copy");
    off += width * W;
  }
  return B3P_OK;
}
}  // namespace

extern "C" {

b3p_status b3p_get_state(b3p_batch *b, b3p_field f, void *dst, size_t bytes, void *stream) {
  return copy_field(b, f, (char *)dst, bytes, false, stream);
}
b3p_status b3p_set_state(b3p_batch *b, b3p_field f, const void *src, size_t bytes, void *stream) {
  if (f == B3P_FIELD_STATS) return fail(B3P_ERR_INVALID_ARG, "stats are read-only");
  return copy_field(b, f, (char *)src, bytes, true, stream);
}

b3p_status b3p_get_contacts(b3p_batch *b, float *dst, size_t bytes, int32_t *count, void *stream) {
  if (!b || ((!dst || !count) && b->total_world > 0)) return fail(B3P_ERR_INVALID_ARG, "null argument");
  if (!b->opt.write_contacts) return fail(B3P_ERR_UNSUPPORTED, "batch created without write_contacts");
  size_t need = 0;
  for (int g = 0; g < (int)b->models.size(); g++) need += (size_t)b->nworld[g] * std::max(b->models[g]->ncon_max, 1) * 24 * 4;
  if (bytes != need) return fail(B3P_ERR_INVALID_ARG, "contacts need %zu bytes, got %zu", need, bytes);
  if (b->total_world == 0) return B3P_OK;
  size_t off = 0, coff = 0;
  for (int g = 0; g < (int)b->models.size(); g++) {
    const DGroup &G = b->host.g[g];
    size_t W = b->nworld[g], n = W * std::max(b->models[g]->ncon_max, 1) * 24 * 4;
    if (W == 0) continue;
    CUDA_TRY(cudaMemcpyAsync((char *)dst + off, G.con, n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "contact copy");
    CUDA_TRY(cudaMemcpyAsync(count + coff, G.ncon, 4 * W, cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "count copy");
    off += n;
    coff += W;
  }
  return B3P_OK;
}

size_t b3p_state_bytes(const b3p_batch *b) { return b ? (size_t)b->state_bytes : 0; }

b3p_status b3p_state_save(b3p_batch *b, void *dst, size_t bytes, void *stream) {
  if (!b || !dst) return fail(B3P_ERR_INVALID_ARG, "null argument");
  if (bytes != b->state_bytes) return fail(B3P_ERR_INVALID_ARG, "state needs %llu bytes", (unsigned long long)b->state_bytes);
  CUDA_TRY(cudaMemcpyAsync(dst, b->base + b->state_off, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "save");
  return B3P_OK;
}

b3p_status b3p_state_restore(b3p_batch *b, const void *src, size_t bytes, void *stream) {
  if (!b || !src) return fail(B3P_ERR_INVALID_ARG, "null argument");
  if (bytes != b->state_bytes) return fail(B3P_ERR_INVALID_ARG, "state needs %llu bytes", (unsigned long long)b->state_bytes);
  CUDA_TRY(cudaMemcpyAsync(b->base + b->state_off, src, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "restore");
  return B3P_OK;
}

}  // extern "C"

extern "C" {

b3p_status b3p_set_idle(b3p_batch *b, const int32_t *world_ids, int32_t n, int32_t idle, void *stream) {
  if (!b) return fail(B3P_ERR_INVALID_ARG, "null batch");
  if (!world_ids) n = b->total_world;
  if (n < 0) return fail(B3P_ERR_INVALID_ARG, "negative count");
  int rc = b3p_launch_idle(b->dev, world_ids, n, idle ? 1 : 0, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "idle launch");
  return B3P_OK;
}

b3p_status b3p_sample_targets(b3p_batch *b, const float *sigma_dev, float *ctrl_dev, void *stream) {
  if (!b || !sigma_dev || !ctrl_dev) return fail(B3P_ERR_INVALID_ARG, "null argument");
  int rc = b3p_launch_targets(b->dev, b->total_world, sigma_dev, ctrl_dev, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "targets launch");
  return B3P_OK;
}

b3p_status b3p_diffik(b3p_batch *b, int32_t group, int32_t body, const float *offset_host,
                      const float *target_pos_dev, const float *target_quat_dev, float lambda, float *ctrl_dev,
                      void *stream) {
  if (!b || !offset_host || !target_pos_dev || !ctrl_dev) return fail(B3P_ERR_INVALID_ARG, "null argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  const b3p_model *m = b->models[group];
  if (body < 1 || body >= m->nb) return fail(B3P_ERR_INVALID_ARG, "body must be a non-world body of the group");
  if (m->nu < 1) return fail(B3P_ERR_INVALID_ARG, "the group has no actuators");
  if (!(lambda > 0.f)) return fail(B3P_ERR_INVALID_ARG, "lambda must be > 0");
  // shared memory per world: the working set, then J [6][nu], the 6 x 6 system and its solution
  int floats = m->smem_floats + 6 * m->nu + 36 + 6;
  int rc = b3p_launch_diffik(b->dev, group, b->nworld[group], floats, body, offset_host[0], offset_host[1],
                             offset_host[2], target_pos_dev, target_quat_dev, lambda, ctrl_dev, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "diffik launch");
  return B3P_OK;
}

b3p_status b3p_raycast(b3p_batch *b, int32_t group, int32_t body, int32_t nray, const float *origins_dev,
                       const float *directions_dev, float max_dist, int32_t world_only, float *dist_dev,
                       void *stream) {
  if (!b || !origins_dev || !directions_dev || !dist_dev || nray < 1) return fail(B3P_ERR_INVALID_ARG, "bad argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  const b3p_model *m = b->models[group];
  if (body < 0 || body >= m->nb) return fail(B3P_ERR_INVALID_ARG, "body out of range");
  if (!(max_dist > 0.f)) return fail(B3P_ERR_INVALID_ARG, "max_dist must be > 0");
  int rc = b3p_launch_raycast(b->dev, group, b->nworld[group], m->smem_floats, body, nray, origins_dev,
                              directions_dev, max_dist, world_only ? 1 : 0, dist_dev, nullptr, nullptr, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "raycast launch");
  return B3P_OK;
}

b3p_status b3p_raycast_hits(b3p_batch *b, int32_t group, int32_t body, int32_t nray, const float *origins_dev,
                            const float *directions_dev, float max_dist, int32_t flags, float *dist_dev,
                            float *pos_dev, float *normal_dev, void *stream) {
  if (!b || !origins_dev || !directions_dev || !dist_dev || nray < 1) return fail(B3P_ERR_INVALID_ARG, "bad argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  if (flags & ~3) return fail(B3P_ERR_INVALID_ARG, "unknown ray-cast flags");
  const b3p_model *m = b->models[group];
  if (body < 0 || body >= m->nb) return fail(B3P_ERR_INVALID_ARG, "body out of range");
  if (!(max_dist > 0.f)) return fail(B3P_ERR_INVALID_ARG, "max_dist must be > 0");
  int rc = b3p_launch_raycast(b->dev, group, b->nworld[group], m->smem_floats, body, nray, origins_dev,
                              directions_dev, max_dist, flags, dist_dev, pos_dev, normal_dev, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "raycast launch");
  return B3P_OK;
}

b3p_status b3p_get_history(b3p_batch *b, int32_t group, int32_t world, float *dst_dev, int32_t *count_dev,
                           void *stream) {
  if (!b || !dst_dev || !count_dev) return fail(B3P_ERR_INVALID_ARG, "null argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  if (world < 0 || world >= b->nworld[group]) return fail(B3P_ERR_INVALID_ARG, "world out of range");
  if (b->opt.history <= 0) return fail(B3P_ERR_UNSUPPORTED, "the batch keeps no history (options.history = 0)");
  int rc = b3p_launch_history(b->dev, group, world, dst_dev, count_dev, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "history launch");
  return B3P_OK;
}

int32_t b3p_observe_width(const b3p_batch *b, int32_t group) {
  if (!b || group < 0 || group >= (int)b->models.size()) return -1;
  const b3p_model *m = b->models[group];
  int nh = 0;
  for (int j = 0; j < m->nj; j++) nh += m->jnt_type[j] != B3P_JNT_FREE;
  return 9 + 2 * nh + m->nu;
}

b3p_status b3p_observe(b3p_batch *b, int32_t group, const float *ctrl_dev, float *out_dev, void *stream) {
  if (!b || !out_dev) return fail(B3P_ERR_INVALID_ARG, "null batch or output");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  int rc = b3p_launch_observe(b->dev, group, b->nworld[group], b3p_observe_width(b, group), ctrl_dev, out_dev, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "observe launch");
  return B3P_OK;
}

b3p_status b3p_contact_sensor(b3p_batch *b, int32_t group, const int32_t *body_ids_dev, int32_t n, float threshold,
                              float dt, float *state_dev, float *force_dev, void *stream) {
  if (!b || !body_ids_dev || !state_dev || !force_dev || n < 1) return fail(B3P_ERR_INVALID_ARG, "bad argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  if (!b->opt.write_contacts) return fail(B3P_ERR_UNSUPPORTED, "the contact sensor needs write_contacts = 1");
  if (!(dt >= 0.f) || !(threshold >= 0.f)) return fail(B3P_ERR_INVALID_ARG, "dt and threshold must be >= 0");
  int rc = b3p_launch_sensor(b->dev, group, b->nworld[group], body_ids_dev, n, threshold, dt, state_dev, force_dev,
                             nullptr, 1, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "sensor launch");
  return B3P_OK;
}

b3p_status b3p_contact_sensor_history(b3p_batch *b, int32_t group, const int32_t *body_ids_dev, int32_t n,
                                      float threshold, float dt, float *state_dev, float *force_dev,
                                      float *history_dev, int32_t depth, void *stream) {
  if (!history_dev || depth < 1) return fail(B3P_ERR_INVALID_ARG, "history needs a buffer and depth >= 1");
  if (!b || !body_ids_dev || !state_dev || !force_dev || n < 1) return fail(B3P_ERR_INVALID_ARG, "bad argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  if (!b->opt.write_contacts) return fail(B3P_ERR_UNSUPPORTED, "the contact sensor needs write_contacts = 1");
  if (!(dt >= 0.f) || !(threshold >= 0.f)) return fail(B3P_ERR_INVALID_ARG, "dt and threshold must be >= 0");
  int rc = b3p_launch_sensor(b->dev, group, b->nworld[group], body_ids_dev, n, threshold, dt, state_dev, force_dev,
                             history_dev, depth, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "sensor launch");
  return B3P_OK;
}

b3p_status b3p_reward(b3p_batch *b, int32_t group, const b3p_reward_cfg *cfg, const float *cmd_dev,
                      const float *action_dev, const float *prev_action_dev, const float *sensor_state_dev,
                      float *reward_dev, float *terms_dev, float *episode_dev, uint32_t *done_dev, void *stream) {
  static_assert(B3P_NTERMS == B3P_REWARD_NTERMS, "term count of the kernel and the ABI");
  if (!b || !cfg || !cmd_dev || !reward_dev || !terms_dev || !episode_dev || !done_dev)
    return fail(B3P_ERR_INVALID_ARG, "null argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  const b3p_model *m = b->models[group];
  if (m->nu > 0 && (!action_dev || !prev_action_dev))
    return fail(B3P_ERR_INVALID_ARG, "the group has actuators: action_dev and prev_action_dev are required");
  if (!(cfg->dt > 0.f)) return fail(B3P_ERR_INVALID_ARG, "dt must be > 0");
  if (!(cfg->sigma_lin > 0.f) || !(cfg->sigma_ang > 0.f)) return fail(B3P_ERR_INVALID_ARG, "sigmas must be > 0");
  static_assert(B3P_NBODYLIST == B3P_REWARD_MAXBODIES, "body-list capacity of the kernel and the ABI");
  if (cfg->nfeet < 0 || cfg->nillegal < 0 || cfg->nfeet > B3P_NBODYLIST || cfg->nillegal > B3P_NBODYLIST)
    return fail(B3P_ERR_INVALID_ARG, "body lists hold 0..%d bodies", B3P_NBODYLIST);
  if (cfg->nfeet > 0 && (!cfg->feet_host || !sensor_state_dev))
    return fail(B3P_ERR_INVALID_ARG, "feet need feet_host and the contact sensor's state");
  if (cfg->nillegal > 0 && !cfg->illegal_host) return fail(B3P_ERR_INVALID_ARG, "illegal_host is null");
  if (cfg->nillegal > 0 && !b->opt.write_contacts)
    return fail(B3P_ERR_UNSUPPORTED, "illegal-contact termination needs write_contacts = 1");
  for (int k = 0; k < cfg->nfeet + cfg->nillegal; k++) {
    int id = k < cfg->nfeet ? cfg->feet_host[k] : cfg->illegal_host[k - cfg->nfeet];
    if (id < 1 || id >= m->nb) return fail(B3P_ERR_INVALID_ARG, "body %d is not a non-world body of the group", id);
  }
  RewardArgs a{};
  for (int k = 0; k < B3P_NTERMS; k++) a.weight[k] = cfg->weight[k];
  a.sigma_lin = cfg->sigma_lin; a.sigma_ang = cfg->sigma_ang; a.air_time_target = cfg->air_time_target;
  a.dt = cfg->dt; a.min_height = cfg->min_base_height; a.max_tilt = cfg->max_tilt;
  a.max_steps = cfg->max_episode_steps; a.nfeet = cfg->nfeet; a.nillegal = cfg->nillegal;
  for (int k = 0; k < cfg->nfeet; k++) a.feet[k] = cfg->feet_host[k];
  for (int k = 0; k < cfg->nillegal; k++) a.illegal[k] = cfg->illegal_host[k];
  a.cmd = cmd_dev; a.action = m->nu > 0 ? action_dev : nullptr; a.prev = m->nu > 0 ? prev_action_dev : nullptr;
  a.sensor = sensor_state_dev;
  a.reward = reward_dev; a.terms = terms_dev; a.episode = episode_dev; a.done = done_dev;
  int rc = b3p_launch_reward(b->dev, group, b->nworld[group], m->smem_floats, &a, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "reward launch");
  return B3P_OK;
}

b3p_status b3p_gather_state(b3p_batch *b, int32_t group, b3p_field f, const int32_t *local_ids_dev, int32_t n,
                            float *dst_dev, void *stream) {
  if (!b || !local_ids_dev || !dst_dev || n < 0) return fail(B3P_ERR_INVALID_ARG, "bad argument");
  if (group < 0 || group >= (int)b->models.size()) return fail(B3P_ERR_INVALID_ARG, "group out of range");
  if (f != B3P_FIELD_QPOS && f != B3P_FIELD_QVEL && f != B3P_FIELD_QACC)
    return fail(B3P_ERR_INVALID_ARG, "gather supports qpos, qvel, qacc");
  int width = f == B3P_FIELD_QPOS ? b->models[group]->nq : b->models[group]->nv;
  int rc = b3p_launch_gather(b->dev, group, (int)f, local_ids_dev, n, width, dst_dev, stream);
  if (rc) return cuda_fail((cudaError_t)rc, "gather launch");
  return B3P_OK;
}

}  // extern "C"

extern "C" {

size_t b3p_plain_workspace_bytes(const b3p_batch *b) {
  if (!b) return 0;
  size_t n = 0;
  for (size_t g = 0; g < b->models.size(); g++) n += (size_t)b->nworld[g] * b->models[g]->smem_floats * 4;
  return n;
}

b3p_status b3p_step_plain(b3p_batch *b, const float *ctrl, int32_t decimation, void *workspace, size_t bytes,
                          void *stream) {
  if (!b) return fail(B3P_ERR_INVALID_ARG, "null batch");
  if (decimation < 1) return fail(B3P_ERR_INVALID_ARG, "decimation must be >= 1");
  size_t need = b3p_plain_workspace_bytes(b);
  if (!workspace || bytes < need)
    return fail(B3P_ERR_WORKSPACE_TOO_SMALL, "plain step needs %zu workspace bytes", need);
  if ((uintptr_t)workspace & 255) return fail(B3P_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  bool need_ctrl = false;
  for (auto *m : b->models) need_ctrl |= m->nu > 0;
  if (need_ctrl && !ctrl) return fail(B3P_ERR_INVALID_ARG, "ctrl is required: a group has actuators");
  char *ws = (char *)workspace;
  for (size_t g = 0; g < b->models.size(); g++) {
    int rc = b3p_launch_plain(b->dev, (int)g, b->nworld[g], ctrl, decimation, (float *)ws,
                              b->models[g]->lim_dof.empty() ? 0 : 1, stream);
    if (rc) return cuda_fail((cudaError_t)rc, "plain step launch");
    ws += (size_t)b->nworld[g] * b->models[g]->smem_floats * 4;
  }
  return B3P_OK;
}

}  // extern "C"

__attribute__((visibility("hidden"))) b3p_status b3p_set_error(b3p_status code, const char *msg) {
  return fail(code, "%s", msg);
}
