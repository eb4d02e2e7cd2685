"""Algorithmic FP32 operation count of one physics substep, per world.

Counts follow the kernels' own arithmetic in the tree-sparse convention: a fused
multiply-add counts 2, an add or multiply 1; square roots, divisions and
trigonometric calls count 1 each (they run on the SFU/FMA pipes as a handful of
instructions). Only work proportional to the physics is counted: index
arithmetic, shuffles and shared-memory traffic are not. Inputs are the model
structure (stored mass-matrix entries, chain lengths, pair types) and the
per-world runtime statistics the step reports (contacts, Newton iterations,
line-search evaluations).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .inputs import BOX, CAPSULE, FREE, HINGE, SPHERE, ModelSpec


@dataclass
class Structure:
    nb: int
    nv: int
    nM: int
    row_len: np.ndarray      # [nv] entries per stored row (dof + ancestors)
    n_hinge: int
    n_slide: int
    n_free: int
    pair_cost: float         # narrow phase of all pairs
    mean_chain: float        # mean chain length of the bodies that carry geoms


def structure(spec: ModelSpec) -> Structure:
    # dof tree: parent of a joint's first dof is the last dof of the nearest ancestor joint
    body_last = {}
    dof_parent = []
    d = 0
    for j, t in enumerate(spec.jnt_type):
        b = int(spec.jnt_body[j])
        p = int(spec.body_parent[b])
        while p > 0 and p not in body_last:
            p = int(spec.body_parent[p])
        first_parent = body_last.get(p, -1) if p > 0 else -1
        n = 6 if t == FREE else 1
        for k in range(n):
            dof_parent.append(first_parent if k == 0 else d - 1)
            d += 1
        body_last[b] = d - 1
    row_len = np.zeros(len(dof_parent), dtype=np.int64)
    for i in range(len(dof_parent)):
        k, n = i, 0
        while k >= 0:
            n += 1
            k = dof_parent[k]
        row_len[i] = n
    cost = {SPHERE: 30.0, CAPSULE: 70.0, BOX: 8 * 24.0 + 60.0}
    pc, chains = 0.0, []
    for g, t in enumerate(spec.geom_type):
        if t in cost and spec.geom_contype[g] | spec.geom_conaffinity[g]:
            pc += cost[int(t)]
            b = int(spec.geom_body[g])
            while b > 0 and b not in body_last:
                b = int(spec.body_parent[b])
            chains.append(row_len[body_last[b]] if b > 0 else 0)
    jt = list(spec.jnt_type)
    return Structure(nb=spec.nbody, nv=len(dof_parent), nM=int(row_len.sum()), row_len=row_len,
                     n_hinge=jt.count(HINGE), n_slide=jt.count(0 + 2), n_free=jt.count(FREE),
                     pair_cost=pc, mean_chain=float(np.mean(chains)) if chains else 0.0)


def ltdl_flops(s: Structure) -> float:
    m = s.row_len - 1
    return float(np.sum(3.0 * m * (m + 1) / 2 + m + 1))


def solve_flops(s: Structure) -> float:
    return 4.0 * (s.nM - s.nv) + s.nv


def smooth_flops(s: Structure) -> float:
    """FK, com quantities, CRBA, LTDL of M, RNE, actuators and the smooth solve."""
    nb, nv = s.nb - 1, s.nv
    fk = 110.0 * nb + 120.0 * s.n_hinge + 40.0 * s.n_slide
    com = 160.0 * nb + 30.0 * nv
    crba = 10.0 * nb + 50.0 * nv + 12.0 * s.nM
    rne = (45.0 * nv + 6.0 * nb) + nb * (36.0 + 36.0 + 30.0 + 12.0) + 6.0 * nb + 12.0 * nv
    act = 5.0 * nv
    return fk + com + crba + ltdl_flops(s) + rne + act + solve_flops(s)


def collide_flops(s: Structure, ncon):
    """Narrow phase of every pair plus the contact rows (impedance, reference, A_nn by
    a chain solve) for one substep."""
    ncon = np.asarray(ncon, dtype=np.float64)
    c = s.mean_chain
    return s.pair_cost + ncon * (c * 21.0 + c * c + 60.0)


def newton_flops(s: Structure, ncon, iters, lsevals):
    """The Newton solve for one substep (array inputs): the start at a_s (J a_s and the
    cone costs there), iterations, line search, final zones. Models whose contacts join two
    trees also weigh the previous acceleration as a start (M a, J a); that is not counted."""
    ncon = np.asarray(ncon, dtype=np.float64)
    iters = np.asarray(iters, dtype=np.float64)
    lsevals = np.asarray(lsevals, dtype=np.float64)
    c = s.mean_chain
    jac = ncon * (12.0 * c + 30.0)                       # J x by chain gather
    matvec = 2.0 * (2 * s.nM - s.nv)
    start = jac + 60.0 * ncon + 2.0 * s.nv
    per_iter = (ncon * (60.0 + 25.0)                     # zones and spatial contact forces
                + ncon * c * 12.0 + 2.0 * s.nv           # gradient J^T f
                + ncon * (48.0 * c + 3.0 * c * (c + 1))  # chain outer products into H
                + ltdl_flops(s) + solve_flops(s)         # factor + solve
                + jac + matvec + 4.0 * s.nv              # J p, M p, dots
                + 6.0 * s.nv + 6.0 * ncon)               # updates
    solve = start + iters * per_iter + lsevals * ncon * 70.0 + ncon * 60.0
    return np.where(ncon > 0, solve, 0.0)


def contact_flops(s: Structure, ncon, iters, lsevals):
    """Collision, contact rows and the Newton solve for one substep (array inputs)."""
    return collide_flops(s, ncon) + newton_flops(s, ncon, iters, lsevals)


def substep_flops(s: Structure, ncon: float, iters_per_substep: float, ls_per_substep: float) -> float:
    integ = 3.0 * s.nv + 40.0 * s.n_free
    return smooth_flops(s) + contact_flops(s, ncon, iters_per_substep, ls_per_substep) + integ


def env_step_flops(spec: ModelSpec, stats: np.ndarray, decimation: int) -> float:
    """Total FLOPs of one environment step over all worlds, from the per-world stats
    [W, 4] (contacts in the last substep, Newton iterations and line-search
    evaluations summed over the step's substeps)."""
    s = structure(spec)
    ncon = stats[:, 0].astype(np.float64)
    it = stats[:, 1].astype(np.float64) / decimation
    ls = stats[:, 3].astype(np.float64) / decimation
    return float(np.sum(substep_flops(s, ncon, it, ls))) * decimation


def stage_flops(spec: ModelSpec, stats: np.ndarray, decimation: int) -> dict:
    """FLOPs of one environment step over all worlds, split like the staged launches
    (kinematics, bias, mass, collide, solve, integrate; load and store move data only).
    Same per-world statistics as env_step_flops."""
    s = structure(spec)
    W = stats.shape[0]
    ncon = stats[:, 0].astype(np.float64)
    it = stats[:, 1].astype(np.float64) / decimation
    ls = stats[:, 3].astype(np.float64) / decimation
    nb, nv = s.nb - 1, s.nv
    kin = 110.0 * nb + 120.0 * s.n_hinge + 40.0 * s.n_slide + 160.0 * nb + 30.0 * nv
    bias = (45.0 * nv + 6.0 * nb) + nb * (36.0 + 36.0 + 30.0 + 12.0) + 6.0 * nb + 12.0 * nv + 5.0 * nv
    mass = 10.0 * nb + 50.0 * nv + 12.0 * s.nM + ltdl_flops(s) + solve_flops(s)
    integ = 3.0 * s.nv + 40.0 * s.n_free
    d = float(decimation)
    return {"load": 0.0, "kinematics": kin * W * d, "bias": bias * W * d, "mass": mass * W * d,
            "collide": float(np.sum(collide_flops(s, ncon))) * d,
            "solve": float(np.sum(newton_flops(s, ncon, it, ls))) * d,
            "integrate": integ * W * d, "store": 0.0}
