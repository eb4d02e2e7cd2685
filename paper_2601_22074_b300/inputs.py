"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmarks.

This module holds no physics: it only describes models (bodies, joints, geoms,
actuators and solver options, as flat numpy arrays) and draws the per-world
parameters and control targets that a run feeds in. Both the FP64 oracle and
the CUDA library derive everything else (dof layout, kinematics, dynamics,
collision pairs) on their own from a `ModelSpec`.

The paper's robots (a humanoid, a quadruped and an arm, from MuJoCo Menagerie,
Section "Tasks") are not available here, so the builders below make synthetic
morphologies with the same degree-of-freedom counts and contact structure:

* `pendulum(3)`   3-link planar hinge chain, capsule links L=0.3 m, r=0.02 m, 1 kg
* `quadruped()`   free base + 4 legs x (hip-abduction, hip, knee); 13 bodies; nv=18
* `humanoid()`    free pelvis + 29 hinges; 30 bodies; nv=35; box feet; capsules
* `manipulation()` 7-hinge arm + 2 slide fingers + free 5 cm cube on a table; nv=15

Conventions: quaternions are (w, x, y, z); the world is body 0; a body has at
most one joint; joint types are FREE=0, HINGE=1, SLIDE=2; geom types are
PLANE=0, SPHERE=1, CAPSULE=2, BOX=3. Geom sizes: sphere (r), capsule (r, half
length along local z), box (half sizes). Inertia is given about the body's
centre of mass in the body frame as (Ixx, Iyy, Izz, Ixy, Ixz, Iyz).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

FREE, HINGE, SLIDE = 0, 1, 2
PLANE, SPHERE, CAPSULE, BOX, HFIELD = 0, 1, 2, 3, 4

# collision classes: (contype & other.conaffinity) | (other.contype & conaffinity)
_ROBOT = dict(contype=1, conaffinity=2)
_GROUND = dict(contype=2, conaffinity=1)
_NONE = dict(contype=0, conaffinity=0)


@dataclasses.dataclass
class Options:
    timestep: float = 0.005
    gravity: Sequence[float] = (0.0, 0.0, -9.81)
    solref: Sequence[float] = (0.02, 1.0)           # timeconst, dampratio
    solimp: Sequence[float] = (0.9, 0.95, 0.001, 0.5, 2.0)  # dmin, dmax, width, mid, power
    newton_iterations: int = 10
    newton_tolerance: float = 1e-6
    ls_iterations: int = 8
    pivot_tau: float = 1e-4
    contact_cap: int = 64
    push_period: int = 0      # env steps between pushes of the first free body (0: off)
    push_sigma: float = 0.0   # std of the planar velocity impulse, m/s


@dataclasses.dataclass
class ModelSpec:
    name: str
    body_parent: np.ndarray
    body_pos: np.ndarray
    body_quat: np.ndarray
    body_mass: np.ndarray
    body_ipos: np.ndarray
    body_inertia: np.ndarray
    jnt_type: np.ndarray
    jnt_body: np.ndarray
    jnt_axis: np.ndarray
    jnt_pos: np.ndarray
    jnt_armature: np.ndarray
    jnt_reset_noise: np.ndarray
    qpos_reset: np.ndarray
    act_jnt: np.ndarray
    act_kp: np.ndarray
    act_kd: np.ndarray
    geom_type: np.ndarray
    geom_body: np.ndarray
    geom_size: np.ndarray
    geom_pos: np.ndarray
    geom_quat: np.ndarray
    geom_contype: np.ndarray
    geom_conaffinity: np.ndarray
    geom_friction: np.ndarray
    opt: Options
    # optional: joint ranges (hinge/slide), DC-motor saturation, actuation delay
    jnt_limited: Optional[np.ndarray] = None     # [njnt] int
    jnt_range: Optional[np.ndarray] = None       # [njnt, 2]
    act_dcmotor: Optional[np.ndarray] = None     # [nu, 3] stall torque, no-load speed, torque limit
    act_delay: int = 0                           # env steps
    # optional heightfield (geoms of type HFIELD on the world body)
    hfield_data: Optional[np.ndarray] = None     # [nrow, ncol] heights, row = y, col = x
    hfield_size: Sequence[float] = (0.0, 0.0)    # half extents x, y

    @property
    def nbody(self) -> int:
        return int(self.body_parent.shape[0])

    @property
    def njnt(self) -> int:
        return int(self.jnt_type.shape[0])

    @property
    def nu(self) -> int:
        return int(self.act_jnt.shape[0])

    @property
    def ngeom(self) -> int:
        return int(self.geom_type.shape[0])

    @property
    def nq(self) -> int:
        return int(sum(7 if t == FREE else 1 for t in self.jnt_type))

    @property
    def nv(self) -> int:
        return int(sum(6 if t == FREE else 1 for t in self.jnt_type))

    def jnt_qposadr(self) -> np.ndarray:
        out, a = [], 0
        for t in self.jnt_type:
            out.append(a)
            a += 7 if t == FREE else 1
        return np.array(out, dtype=np.int32)

    def jnt_dofadr(self) -> np.ndarray:
        out, a = [], 0
        for t in self.jnt_type:
            out.append(a)
            a += 6 if t == FREE else 1
        return np.array(out, dtype=np.int32)

    def act_qposadr(self) -> np.ndarray:
        qa = self.jnt_qposadr()
        return np.array([qa[j] for j in self.act_jnt], dtype=np.int32)

    def replace_opt(self, **kw) -> "ModelSpec":
        return dataclasses.replace(self, opt=dataclasses.replace(self.opt, **kw))


# --------------------------------------------------------------------------- inertia of shapes
def sphere_inertia(m: float, r: float):
    i = 0.4 * m * r * r
    return (i, i, i, 0.0, 0.0, 0.0)


def cylinder_inertia_z(m: float, r: float, length: float):
    """Solid cylinder of radius r and length `length` along the local z axis."""
    ia = 0.5 * m * r * r
    it = m * (3.0 * r * r + length * length) / 12.0
    return (it, it, ia, 0.0, 0.0, 0.0)


def cylinder_inertia_y(m: float, r: float, length: float):
    ia = 0.5 * m * r * r
    it = m * (3.0 * r * r + length * length) / 12.0
    return (it, ia, it, 0.0, 0.0, 0.0)


def box_inertia(m: float, half: Sequence[float]):
    a, b, c = (2.0 * h for h in half)
    return (m * (b * b + c * c) / 12.0, m * (a * a + c * c) / 12.0,
            m * (a * a + b * b) / 12.0, 0.0, 0.0, 0.0)


_QX90 = (math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0)  # local z -> world -y


class _Builder:
    def __init__(self, name: str):
        self.name = name
        self.b: Dict[str, List] = {k: [] for k in
                                   ("parent", "pos", "quat", "mass", "ipos", "inertia")}
        self.j: Dict[str, List] = {k: [] for k in
                                   ("type", "body", "axis", "pos", "armature", "noise")}
        self.g: Dict[str, List] = {k: [] for k in ("type", "body", "size", "pos", "quat",
                                                   "contype", "conaffinity", "friction")}
        self.a: Dict[str, List] = {k: [] for k in ("jnt", "kp", "kd")}
        self.qpos_reset: List[float] = []
        self.body(-1, (0, 0, 0))  # world

    def body(self, parent, pos, quat=(1, 0, 0, 0), mass=0.0, ipos=(0, 0, 0),
             inertia=(0, 0, 0, 0, 0, 0)) -> int:
        self.b["parent"].append(parent)
        self.b["pos"].append(pos)
        self.b["quat"].append(quat)
        self.b["mass"].append(mass)
        self.b["ipos"].append(ipos)
        self.b["inertia"].append(inertia)
        return len(self.b["parent"]) - 1

    def joint(self, body, jtype, axis=(0, 0, 1), pos=(0, 0, 0), armature=0.0,
              reset=0.0, noise=0.0) -> int:
        self.j["type"].append(jtype)
        self.j["body"].append(body)
        self.j["axis"].append(axis)
        self.j["pos"].append(pos)
        self.j["armature"].append(armature)
        self.j["noise"].append(noise)
        if jtype == FREE:
            self.qpos_reset.extend(list(self.b["pos"][body]) + list(self.b["quat"][body]))
        else:
            self.qpos_reset.append(reset)
        return len(self.j["type"]) - 1

    def geom(self, body, gtype, size, pos=(0, 0, 0), quat=(1, 0, 0, 0), friction=1.0,
             contype=0, conaffinity=0) -> int:
        s = list(size) + [0.0] * (3 - len(size))
        self.g["type"].append(gtype)
        self.g["body"].append(body)
        self.g["size"].append(s)
        self.g["pos"].append(pos)
        self.g["quat"].append(quat)
        self.g["contype"].append(contype)
        self.g["conaffinity"].append(conaffinity)
        self.g["friction"].append(friction)
        return len(self.g["type"]) - 1

    def actuator(self, jnt, kp, kd) -> int:
        self.a["jnt"].append(jnt)
        self.a["kp"].append(kp)
        self.a["kd"].append(kd)
        return len(self.a["jnt"]) - 1

    def build(self, opt: Options) -> ModelSpec:
        f64 = lambda x, shape: np.asarray(x, dtype=np.float64).reshape(shape)
        i32 = lambda x: np.asarray(x, dtype=np.int32).reshape(-1)
        u32 = lambda x: np.asarray(x, dtype=np.uint32).reshape(-1)
        nb, nj, ng, nu = (len(self.b["parent"]), len(self.j["type"]),
                          len(self.g["type"]), len(self.a["jnt"]))
        return ModelSpec(
            name=self.name,
            body_parent=i32(self.b["parent"]),
            body_pos=f64(self.b["pos"], (nb, 3)),
            body_quat=f64(self.b["quat"], (nb, 4)),
            body_mass=f64(self.b["mass"], (nb,)),
            body_ipos=f64(self.b["ipos"], (nb, 3)),
            body_inertia=f64(self.b["inertia"], (nb, 6)),
            jnt_type=i32(self.j["type"]),
            jnt_body=i32(self.j["body"]),
            jnt_axis=f64(self.j["axis"], (nj, 3)),
            jnt_pos=f64(self.j["pos"], (nj, 3)),
            jnt_armature=f64(self.j["armature"], (nj,)),
            jnt_reset_noise=f64(self.j["noise"], (nj,)),
            qpos_reset=f64(self.qpos_reset, (-1,)),
            act_jnt=i32(self.a["jnt"]),
            act_kp=f64(self.a["kp"], (nu,)),
            act_kd=f64(self.a["kd"], (nu,)),
            geom_type=i32(self.g["type"]),
            geom_body=i32(self.g["body"]),
            geom_size=f64(self.g["size"], (ng, 3)),
            geom_pos=f64(self.g["pos"], (ng, 3)),
            geom_quat=f64(self.g["quat"], (ng, 4)),
            geom_contype=u32(self.g["contype"]),
            geom_conaffinity=u32(self.g["conaffinity"]),
            geom_friction=f64(self.g["friction"], (ng,)),
            opt=opt,
        )


# --------------------------------------------------------------------------- morphologies
def pendulum(nlink: int = 3, length: float = 0.3, radius: float = 0.02, mass: float = 1.0,
             noise: float = math.pi, timestep: float = 0.002, nchain: int = 1, **optkw) -> ModelSpec:
    """Planar hinge chain hanging from the world origin along -z at q=0; axes along y.

    Each link: a solid-cylinder capsule of length `length`, centre of mass at L/2.
    No contacts and no actuators (configuration "64 worlds of a 3-link pendulum").
    nchain > 1: that many such chains, hung 0.5 m apart along x (a large tree-sparse model:
    two chains of 31 links have nv = 62 and 63 bodies, near the limits of 64 of each).
    """
    bld = _Builder(f"pendulum{nlink}" if nchain == 1 else f"pendulum{nchain}x{nlink}")
    for c in range(nchain):
        parent = 0
        for i in range(nlink):
            pos = (0.5 * c, 0, 0) if i == 0 else (0, 0, -length)
            b = bld.body(parent, pos, mass=mass, ipos=(0, 0, -length / 2),
                         inertia=cylinder_inertia_z(mass, radius, length))
            bld.joint(b, HINGE, axis=(0, 1, 0), noise=noise)
            bld.geom(b, CAPSULE, (radius, length / 2), pos=(0, 0, -length / 2), **_NONE)
            parent = b
    return bld.build(Options(timestep=timestep, **optkw))


def quadruped(**optkw) -> ModelSpec:
    """Free base box 0.4x0.2x0.1 m (6 kg) with 4 legs x (hip-abduction x, hip y, knee y).

    Thigh and calf are capsules 0.2 m long, r=0.02 (1 kg, 0.5 kg); a sphere foot
    r=0.02 sits at the end of the calf. Default pose hip=0.6, knee=-1.2 rad, base
    height such that the feet start 5 mm above the plane z=0.
    """
    bld = _Builder("quadruped")
    bld.geom(0, PLANE, (0, 0, 0), **_GROUND)
    base_z = 0.4 * math.cos(0.6) + 0.02 + 0.005
    half = (0.2, 0.1, 0.05)
    base = bld.body(0, (0, 0, base_z), mass=6.0, inertia=box_inertia(6.0, half))
    bld.joint(base, FREE)
    bld.geom(base, BOX, half, **_ROBOT)
    for sx, sy in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
        hip = bld.body(base, (0.18 * sx, 0.12 * sy, 0.0), mass=0.3,
                       inertia=sphere_inertia(0.3, 0.04))
        j = bld.joint(hip, HINGE, axis=(1, 0, 0), armature=0.01, noise=0.05)
        bld.actuator(j, 40.0, 1.0)
        thigh = bld.body(hip, (0, 0.05 * sy, 0), mass=1.0, ipos=(0, 0, -0.1),
                         inertia=cylinder_inertia_z(1.0, 0.02, 0.2))
        j = bld.joint(thigh, HINGE, axis=(0, 1, 0), armature=0.01, reset=0.6, noise=0.05)
        bld.actuator(j, 40.0, 1.0)
        bld.geom(thigh, CAPSULE, (0.02, 0.1), pos=(0, 0, -0.1), **_ROBOT)
        calf = bld.body(thigh, (0, 0, -0.2), mass=0.5, ipos=(0, 0, -0.1),
                        inertia=cylinder_inertia_z(0.5, 0.02, 0.2))
        j = bld.joint(calf, HINGE, axis=(0, 1, 0), armature=0.01, reset=-1.2, noise=0.05)
        bld.actuator(j, 40.0, 1.0)
        bld.geom(calf, CAPSULE, (0.02, 0.1), pos=(0, 0, -0.1), **_ROBOT)
        bld.geom(calf, SPHERE, (0.02,), pos=(0, 0, -0.2), **_ROBOT)
    opt = dict(timestep=0.005)
    opt.update(optkw)
    return bld.build(Options(**opt))


def humanoid(**optkw) -> ModelSpec:
    """Free pelvis + 29 hinges: legs 2x6, waist 3, arms 2x7 (30 bodies, nv=35, nq=36).

    Box feet 0.2x0.08x0.03 m; capsules for pelvis, torso, thighs, shins, upper arms and
    forearms; spheres for head and hands; self-collision off (robot geoms only
    collide with the ground plane). The longest ancestor chain has 16 dofs and the
    tree-sparse mass matrix has 341 stored entries.
    """
    bld = _Builder("humanoid")
    bld.geom(0, PLANE, (0, 0, 0), **_GROUND)
    small = lambda m: dict(mass=m, inertia=sphere_inertia(m, 0.04))
    X, Y, Z = (1, 0, 0), (0, 1, 0), (0, 0, 1)
    arm, noise = 0.01, 0.05
    acts = []

    def hinge(body, axis):
        acts.append(bld.joint(body, HINGE, axis=axis, armature=arm, noise=noise))

    pelvis = bld.body(0, (0, 0, 0.735), mass=5.0, inertia=cylinder_inertia_y(5.0, 0.07, 0.3))
    bld.joint(pelvis, FREE)
    bld.geom(pelvis, CAPSULE, (0.07, 0.08), quat=_QX90, **_ROBOT)
    for sy in (1, -1):
        hp = bld.body(pelvis, (0, 0.1 * sy, -0.08), **small(1.0)); hinge(hp, Y)
        hr = bld.body(hp, (0, 0, 0), **small(1.0)); hinge(hr, X)
        th = bld.body(hr, (0, 0, 0), mass=3.0, ipos=(0, 0, -0.15),
                      inertia=cylinder_inertia_z(3.0, 0.05, 0.3)); hinge(th, Z)
        bld.geom(th, CAPSULE, (0.05, 0.12), pos=(0, 0, -0.15), **_ROBOT)
        sh = bld.body(th, (0, 0, -0.3), mass=2.0, ipos=(0, 0, -0.15),
                      inertia=cylinder_inertia_z(2.0, 0.04, 0.3)); hinge(sh, Y)
        bld.geom(sh, CAPSULE, (0.04, 0.12), pos=(0, 0, -0.15), **_ROBOT)
        ap = bld.body(sh, (0, 0, -0.3), **small(0.3)); hinge(ap, Y)
        foot_half = (0.1, 0.04, 0.015)
        ft = bld.body(ap, (0, 0, 0), mass=0.7, ipos=(0.03, 0, -0.035),
                      inertia=box_inertia(0.7, foot_half)); hinge(ft, X)
        bld.geom(ft, BOX, foot_half, pos=(0.03, 0, -0.035), **_ROBOT)
    wy = bld.body(pelvis, (0, 0, 0.05), **small(1.0)); hinge(wy, Z)
    wr = bld.body(wy, (0, 0, 0), **small(1.0)); hinge(wr, X)
    torso = bld.body(wr, (0, 0, 0), mass=8.0, ipos=(0, 0, 0.2),
                     inertia=cylinder_inertia_z(8.0, 0.09, 0.3)); hinge(torso, Y)
    bld.geom(torso, CAPSULE, (0.09, 0.15), pos=(0, 0, 0.2), **_ROBOT)
    bld.geom(torso, SPHERE, (0.09,), pos=(0, 0, 0.5), **_ROBOT)
    for sy in (1, -1):
        sp = bld.body(torso, (0, 0.2 * sy, 0.33), **small(0.5)); hinge(sp, Y)
        sr = bld.body(sp, (0, 0, 0), **small(0.5)); hinge(sr, X)
        ua = bld.body(sr, (0, 0, 0), mass=1.0, ipos=(0, 0, -0.125),
                      inertia=cylinder_inertia_z(1.0, 0.035, 0.25)); hinge(ua, Z)
        bld.geom(ua, CAPSULE, (0.035, 0.1), pos=(0, 0, -0.125), **_ROBOT)
        fa = bld.body(ua, (0, 0, -0.25), mass=0.6, ipos=(0, 0, -0.11),
                      inertia=cylinder_inertia_z(0.6, 0.03, 0.22)); hinge(fa, Y)
        bld.geom(fa, CAPSULE, (0.03, 0.09), pos=(0, 0, -0.11), **_ROBOT)
        wrr = bld.body(fa, (0, 0, -0.22), **small(0.2)); hinge(wrr, X)
        wrp = bld.body(wrr, (0, 0, 0), **small(0.2)); hinge(wrp, Y)
        hand = bld.body(wrp, (0, 0, 0), mass=0.3, ipos=(0, 0, -0.04),
                        inertia=sphere_inertia(0.3, 0.04)); hinge(hand, Z)
        bld.geom(hand, SPHERE, (0.04,), pos=(0, 0, -0.04), **_ROBOT)
    for j in acts:
        bld.actuator(j, 100.0, 2.0)
    opt = dict(timestep=0.005, push_period=200, push_sigma=0.5)
    opt.update(optkw)
    return bld.build(Options(**opt))


def manipulation(base_z: float = 0.42, finger_y: float = 0.045, cube_x: float = 0.45,
                 arm_kp: float = 50.0, arm_kd: float = 2.0, **optkw) -> ModelSpec:
    """7-hinge capsule arm on a world-fixed table box, 2 slide fingers (boxes), free cube.

    The cube (5 cm, 0.1 kg) rests on the table; the open gripper starts 2 cm above it.
    Contacts are box-box (cube-table and cube-finger). Arm links do not collide.
    nq=16, nv=15, nu=9.
    """
    bld = _Builder("manipulation")
    bld.geom(0, PLANE, (0, 0, 0), **_GROUND)   # the floor, for cubes knocked off the table
    table_half = (0.4, 0.4, 0.2)
    bld.geom(0, BOX, table_half, pos=(0.45, 0, 0.2), contype=2, conaffinity=1)
    axes = [(0, 0, 1), (0, 1, 0), (0, 0, 1), (0, 1, 0), (0, 0, 1), (0, 1, 0), (0, 0, 1)]
    lens = [0.1, 0.25, 0.05, 0.25, 0.05, 0.1, 0.05]
    reset = [0.0, 0.6, 0.0, 1.2, 0.0, 1.3, 0.0]
    parent, pos = 0, (0.0, 0.0, base_z)
    acts = []
    for k in range(7):
        m = 1.5 - 0.15 * k
        b = bld.body(parent, pos, mass=m, ipos=(0, 0, lens[k] / 2),
                     inertia=cylinder_inertia_z(m, 0.04, max(lens[k], 0.08)))
        acts.append((bld.joint(b, HINGE, axis=axes[k], armature=0.01, reset=reset[k],
                               noise=0.05), arm_kp, arm_kd))
        bld.geom(b, CAPSULE, (0.04, lens[k] / 2), pos=(0, 0, lens[k] / 2), **_NONE)
        parent, pos = b, (0, 0, lens[k])
    for sy in (1, -1):
        f_half = (0.01, 0.01, 0.04)
        f = bld.body(parent, (0, finger_y * sy, 0.05), mass=0.05, ipos=(0, 0, 0.04),
                     inertia=box_inertia(0.05, f_half))
        acts.append((bld.joint(f, SLIDE, axis=(0, sy, 0), armature=0.01, reset=0.0,
                               noise=0.005), 200.0, 2.0))
        bld.geom(f, BOX, f_half, pos=(0, 0, 0.04), contype=4, conaffinity=0)
    cube_half = (0.025, 0.025, 0.025)
    cube = bld.body(0, (cube_x, 0.0, 0.4 + 0.025), mass=0.1, inertia=box_inertia(0.1, cube_half))
    bld.joint(cube, FREE)
    bld.geom(cube, BOX, cube_half, contype=1, conaffinity=2 | 4)
    for j, kp, kd in acts:
        bld.actuator(j, kp, kd)
    opt = dict(timestep=0.005)
    opt.update(optkw)
    return bld.build(Options(**opt))


def free_body(shape: int = SPHERE, size=(0.1,), mass: float = 1.0, pos=(0, 0, 1.0),
              quat=(1, 0, 0, 0), inertia=None, plane: bool = True, friction: float = 1.0,
              timestep: float = 0.005, **optkw) -> ModelSpec:
    """One free body (sphere/capsule/box) above an optional ground plane: test fixtures."""
    bld = _Builder("free_body")
    if plane:
        bld.geom(0, PLANE, (0, 0, 0), friction=friction, **_GROUND)
    if inertia is None:
        if shape == SPHERE:
            inertia = sphere_inertia(mass, size[0])
        elif shape == BOX:
            inertia = box_inertia(mass, size)
        else:
            inertia = cylinder_inertia_z(mass, size[0], 2 * size[1])
    b = bld.body(0, pos, quat=quat, mass=mass, inertia=inertia)
    bld.joint(b, FREE)
    bld.geom(b, shape, size, friction=friction, **_ROBOT)
    return bld.build(Options(timestep=timestep, **optkw))


def spatial_chain(timestep: float = 0.002, **optkw) -> ModelSpec:
    """Fixed-base test chain mixing hinge x/z/y and slide joints, rotated body frames,
    off-axis joint anchors and off-centre masses (exercises every kinematic term)."""
    bld = _Builder("spatial_chain")
    c, s = math.cos(0.3), math.sin(0.3)
    b1 = bld.body(0, (0.1, 0.0, 0.5), quat=(c, 0, s, 0), mass=1.2, ipos=(0.02, 0.01, -0.1),
                  inertia=(0.02, 0.015, 0.01, 0.001, -0.002, 0.0005))
    bld.joint(b1, HINGE, axis=(1, 0, 0), pos=(0.0, 0.02, 0.0), noise=0.5)
    b2 = bld.body(b1, (0.0, 0.1, -0.2), quat=(c, s, 0, 0), mass=0.8, ipos=(0.0, 0.05, -0.05),
                  inertia=(0.01, 0.012, 0.006, 0.0, 0.001, 0.0))
    bld.joint(b2, HINGE, axis=(0, 0.6, 0.8), pos=(0.01, 0.0, 0.03), noise=0.5)
    b3 = bld.body(b2, (0.05, 0.0, -0.15), mass=0.5, ipos=(0.0, 0.0, -0.05),
                  inertia=(0.004, 0.004, 0.002, 0.0, 0.0, 0.0))
    bld.joint(b3, SLIDE, axis=(0, 1, 0), noise=0.05)
    b4 = bld.body(b3, (0.0, 0.0, -0.1), quat=(c, 0, 0, s), mass=0.6, ipos=(0.03, 0.0, -0.08),
                  inertia=(0.005, 0.006, 0.003, 0.0002, 0.0, 0.0))
    bld.joint(b4, HINGE, axis=(0, 1, 0), pos=(0.0, 0.0, 0.0), noise=0.5)
    b5 = bld.body(b4, (0.0, 0.05, -0.2), mass=0.4, ipos=(0.0, 0.0, -0.04),
                  inertia=(0.002, 0.002, 0.001, 0.0, 0.0, 0.0))
    bld.joint(b5, HINGE, axis=(0, 0, 1), noise=0.5)
    return bld.build(Options(timestep=timestep, **optkw))


MORPHOLOGIES = {
    "pendulum": pendulum,
    "quadruped": quadruped,
    "humanoid": humanoid,
    "manipulation": manipulation,
}


# --------------------------------------------------------------------------- per-world inputs
@dataclasses.dataclass
class WorldParams:
    """Per-world domain-randomised fields (float64 host arrays)."""
    friction_scale: np.ndarray   # [W]
    mass_scale: np.ndarray       # [W, nbody]
    kp: np.ndarray               # [W, nu]
    kd: np.ndarray               # [W, nu]
    inertia: Optional[np.ndarray] = None   # [W, nbody, 10] mass, com (3), inertia (6); None: model


def default_params(spec: ModelSpec, nworld: int) -> WorldParams:
    return WorldParams(
        friction_scale=np.ones(nworld),
        mass_scale=np.ones((nworld, spec.nbody)),
        kp=np.tile(spec.act_kp, (nworld, 1)),
        kd=np.tile(spec.act_kd, (nworld, 1)),
    )


def randomised_params(spec: ModelSpec, nworld: int, seed: int) -> WorldParams:
    """Domain randomisation recipes of the benchmark configurations.

    quadruped: friction ~ U[0.3, 1.2] per world, link mass scale ~ U[0.8, 1.2] per link.
    humanoid: kp ~ U[50, 150] per actuator per world, kd = 0.02 kp.
    manipulation, pendulum: model defaults.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    p = default_params(spec, nworld)
    if spec.name == "quadruped":
        p.friction_scale = rng.uniform(0.3, 1.2, size=nworld)
        p.mass_scale[:, 1:] = rng.uniform(0.8, 1.2, size=(nworld, spec.nbody - 1))
    elif spec.name == "humanoid":
        p.kp = rng.uniform(50.0, 150.0, size=(nworld, spec.nu))
        p.kd = 0.02 * p.kp
    return p


CTRL_SIGMA = {"pendulum": 0.0, "quadruped": 0.5, "humanoid": 0.3, "manipulation": 0.3}


def ctrl_targets(spec: ModelSpec, nworld: int, nsteps: int, seed: int,
                 sigma: Optional[float] = None) -> np.ndarray:
    """PD position targets [nsteps, W, nu]: the default pose plus N(0, sigma) rad."""
    if sigma is None:
        sigma = CTRL_SIGMA.get(spec.name, 0.3)
    rng = np.random.Generator(np.random.PCG64(seed))
    center = spec.qpos_reset[spec.act_qposadr()]
    noise = rng.normal(0.0, 1.0, size=(nsteps, nworld, spec.nu)) * sigma
    return (center[None, None, :] + noise).astype(np.float64)


# --------------------------------------------------------------------------- benchmark configs
@dataclasses.dataclass
class Workload:
    name: str
    groups: List[tuple]   # (morphology name, nworld)
    decimation: int
    steps: int


WORKLOADS = {
    "pendulum64": Workload("pendulum64", [("pendulum", 64)], 1, 1000),
    "quadruped4096": Workload("quadruped4096", [("quadruped", 4096)], 4, 100),
    "humanoid8192": Workload("humanoid8192", [("humanoid", 8192)], 4, 100),
    "hetero9216": Workload("hetero9216", [("pendulum", 2048), ("quadruped", 4096),
                                          ("humanoid", 2048), ("manipulation", 1024)], 4, 100),
}


# ---------------------------------------------------------------- actuator / limit variants
def with_limits(spec: ModelSpec, half_range: float = 0.3, joints: Optional[Sequence[int]] = None) -> ModelSpec:
    """Range [reset - half_range, reset + half_range] on every hinge/slide joint (or the
    listed ones), enforced by limit rows in the constraint solve."""
    qa = spec.jnt_qposadr()
    lim = np.zeros(spec.njnt, dtype=np.int32)
    rng = np.zeros((spec.njnt, 2))
    for j, t in enumerate(spec.jnt_type):
        if t == FREE or (joints is not None and j not in joints):
            continue
        lim[j] = 1
        rng[j] = (spec.qpos_reset[qa[j]] - half_range, spec.qpos_reset[qa[j]] + half_range)
    return dataclasses.replace(spec, name=spec.name + "_lim", jnt_limited=lim, jnt_range=rng)


def with_dcmotor(spec: ModelSpec, stall: float, no_load_speed: float, limit: float) -> ModelSpec:
    """The same DC-motor torque-speed line on every actuator."""
    dc = np.tile(np.array([[stall, no_load_speed, limit]], dtype=np.float64), (spec.nu, 1))
    return dataclasses.replace(spec, name=spec.name + "_dc", act_dcmotor=dc)


def with_delay(spec: ModelSpec, steps: int) -> ModelSpec:
    """Actuation delay of `steps` env steps."""
    return dataclasses.replace(spec, name=spec.name + f"_d{steps}", act_delay=int(steps))


def with_terrain(spec: ModelSpec, nrow: int = 41, ncol: int = 41, half: float = 2.0, amplitude: float = 0.04,
                 seed: int = 0) -> ModelSpec:
    """Replace the ground plane by a heightfield of the same extent around the origin:
    random bumps (a sum of seeded Gaussian hills of height up to `amplitude`) on an
    nrow x ncol grid of half extent `half` (section "Components": terrain)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = np.linspace(-half, half, ncol)
    ys = np.linspace(-half, half, nrow)
    X, Y = np.meshgrid(xs, ys)
    Z = np.zeros_like(X)
    for _ in range(24):
        cx, cy = rng.uniform(-half, half, 2)
        w = rng.uniform(0.2, 0.6)
        Z += rng.uniform(-1.0, 1.0) * amplitude * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * w * w))
    gt = spec.geom_type.copy()
    planes = np.where((gt == PLANE) & (spec.geom_body == 0))[0]
    assert len(planes) >= 1, "the model has no ground plane"
    gt[planes[0]] = HFIELD
    return dataclasses.replace(spec, name=spec.name + "_terrain", geom_type=gt, hfield_data=Z,
                               hfield_size=(half, half))


# ---------------------------------------------------------------- inertia randomisation
# Pseudo-inertia J = [[S, h], [h^T, m]] with h = m c, S = tr(Ibar)/2 1 - Ibar, Ibar the
# rotational inertia about the body origin; J is positive definite exactly for physically
# consistent (m, c, I) (Wensing et al.). Its log-Cholesky factor J = U U^T,
# U = e^a [[e^d1, s12, s13, t1], [0, e^d2, s23, t2], [0, 0, e^d3, t3], [0, 0, 0, 1]], maps
# the unconstrained vector (a, d1, d2, d3, s12, s23, s13, t1, t2, t3) onto consistent
# inertias (Rucker and Wensing, "Smooth parameterization of rigid-body inertia"), so
# randomising that vector keeps every sample physical (section "Manager-Based API":
# domain randomisation with pseudo-inertia consistency).
def inertia_to_pseudo(mass, com, inertia6):
    c = np.asarray(com, dtype=np.float64)
    Ixx, Iyy, Izz, Ixy, Ixz, Iyz = inertia6
    Ic = np.array([[Ixx, Ixy, Ixz], [Ixy, Iyy, Iyz], [Ixz, Iyz, Izz]])
    Ibar = Ic + mass * (c @ c * np.eye(3) - np.outer(c, c))
    J = np.zeros((4, 4))
    J[:3, :3] = 0.5 * np.trace(Ibar) * np.eye(3) - Ibar
    J[:3, 3] = J[3, :3] = mass * c
    J[3, 3] = mass
    return J


def pseudo_to_inertia(J):
    mass = J[3, 3]
    c = J[:3, 3] / mass
    S = J[:3, :3]
    Ibar = np.trace(S) * np.eye(3) - S
    Ic = Ibar - mass * (c @ c * np.eye(3) - np.outer(c, c))
    return mass, c, np.array([Ic[0, 0], Ic[1, 1], Ic[2, 2], Ic[0, 1], Ic[0, 2], Ic[1, 2]])


def pseudo_to_logchol(J):
    P = np.eye(4)[::-1]
    U = P @ np.linalg.cholesky(P @ J @ P) @ P     # upper triangular, J = U U^T
    a = np.log(U[3, 3])
    V = U / U[3, 3]
    return np.array([a, np.log(V[0, 0]), np.log(V[1, 1]), np.log(V[2, 2]), V[0, 1], V[1, 2], V[0, 2],
                     V[0, 3], V[1, 3], V[2, 3]])


def logchol_to_pseudo(theta):
    a, d1, d2, d3, s12, s23, s13, t1, t2, t3 = theta
    U = np.exp(a) * np.array([[np.exp(d1), s12, s13, t1], [0, np.exp(d2), s23, t2],
                              [0, 0, np.exp(d3), t3], [0, 0, 0, 1.0]])
    return U @ U.T


def randomised_inertia(spec: ModelSpec, nworld: int, seed: int, sigma: float = 0.1) -> np.ndarray:
    """[W, nbody, 10] per-world body inertias: each moving body's log-Cholesky vector
    perturbed by N(0, sigma^2) per component (the world body stays massless)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((nworld, spec.nbody, 10))
    for b in range(spec.nbody):
        base = np.concatenate([[spec.body_mass[b]], spec.body_ipos[b], spec.body_inertia[b]])
        out[:, b] = base
        if b == 0 or spec.body_mass[b] <= 0:
            continue
        th = pseudo_to_logchol(inertia_to_pseudo(spec.body_mass[b], spec.body_ipos[b], spec.body_inertia[b]))
        for w in range(nworld):
            m, c, I6 = pseudo_to_inertia(logchol_to_pseudo(th + sigma * rng.normal(size=10)))
            out[w, b] = np.concatenate([[m], c, I6])
    return out
