"""ctypes wrapper of the FP64 oracle library (oracle.cpp). Test infrastructure only.

`Oracle(spec)` compiles nothing by itself: call `build_oracle()` first (the
`__graft_entry__.build()` step and the test session do it).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
CON_STRIDE = 24

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint32)


class _Desc(C.Structure):
    _fields_ = [
        ("nbody", C.c_int32), ("njnt", C.c_int32), ("nu", C.c_int32), ("ngeom", C.c_int32),
        ("body_parent", _ip),
        ("body_pos", _dp), ("body_quat", _dp), ("body_mass", _dp), ("body_ipos", _dp),
        ("body_inertia", _dp),
        ("jnt_type", _ip), ("jnt_body", _ip),
        ("jnt_axis", _dp), ("jnt_pos", _dp), ("jnt_armature", _dp), ("jnt_reset_noise", _dp),
        ("qpos_reset", _dp),
        ("act_jnt", _ip), ("act_kp", _dp), ("act_kd", _dp),
        ("geom_type", _ip), ("geom_body", _ip),
        ("geom_size", _dp), ("geom_pos", _dp), ("geom_quat", _dp),
        ("geom_contype", _up), ("geom_conaffinity", _up), ("geom_friction", _dp),
        ("timestep", C.c_double), ("gravity", C.c_double * 3), ("solref", C.c_double * 2),
        ("solimp", C.c_double * 5), ("newton_iterations", C.c_int32),
        ("newton_tolerance", C.c_double), ("ls_iterations", C.c_int32),
        ("pivot_tau", C.c_double), ("contact_cap", C.c_int32), ("push_period", C.c_int32),
        ("push_sigma", C.c_double),
        ("jnt_limited", _ip), ("jnt_range", _dp), ("act_dcmotor", _dp),
        ("hfield_nrow", C.c_int32), ("hfield_ncol", C.c_int32), ("hfield_size", C.c_double * 2),
        ("hfield_data", _dp),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (g++ -O2, FP64, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
           "-Wall", "-o", _LIB + ".tmp", _SRC]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def build_oracle_sanitized() -> str:
    """The oracle built with AddressSanitizer and UndefinedBehaviorSanitizer (for the
    host-memory check of the tests; load it with ORACLE_LIB set and libasan preloaded)."""
    out = os.path.join(_HERE, "liboracle_asan.so")
    cmd = ["g++", "-O1", "-g", "-std=c++17", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer",
           "-o", out + ".tmp", _SRC]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


def _load():
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIB", _LIB)
        if path == _LIB and not os.path.exists(_LIB):
            build_oracle()
        lib = C.CDLL(path)
        lib.orc_model_create.restype = C.c_void_p
        lib.orc_model_create.argtypes = [C.POINTER(_Desc), C.c_char_p, C.c_int]
        lib.orc_model_destroy.argtypes = [C.c_void_p]
        lib.orc_model_info.argtypes = [C.c_void_p, _ip]
        lib.orc_model_pairs.argtypes = [C.c_void_p, _ip]
        lib.orc_philox.argtypes = [_up, _up, _up]
        lib.orc_fk.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.orc_mass_matrix.argtypes = [C.c_void_p, _dp, _dp, _dp]
        lib.orc_rne.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int, _dp, _dp]
        lib.orc_ltdl.argtypes = [C.c_void_p, _dp, _dp, _dp]
        lib.orc_ltdl.restype = C.c_int
        lib.orc_ltdl_solve.argtypes = [C.c_void_p, _dp, _dp, _dp]
        lib.orc_collide.argtypes = [C.c_void_p, _dp, _dp, C.c_int]
        lib.orc_collide.restype = C.c_int
        lib.orc_constraints.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_double, _dp, C.c_int,
                                        _dp, _dp, _dp, _dp]
        lib.orc_constraints.restype = C.c_int
        lib.orc_box_box.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, C.c_int, _ip, _dp]
        lib.orc_box_box.restype = C.c_int
        lib.orc_limits.argtypes = [C.c_void_p, _dp, _dp, _dp, _ip, _dp, _dp, _dp, _dp, C.c_int]
        lib.orc_limits.restype = C.c_int
        lib.orc_cost.argtypes = [C.c_int, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp, C.c_int, _dp,
                                 _dp, _dp, _dp]
        lib.orc_cost.restype = C.c_double
        lib.orc_newton.argtypes = [C.c_int, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp, C.c_int, _dp,
                                   _dp, _dp, _dp, _dp, _dp, _dp, C.c_int]
        lib.orc_newton.restype = C.c_int
        lib.orc_reset.argtypes = [C.c_void_p, C.c_uint64, C.c_int32, _dp, _dp]
        lib.orc_body_jacobian.argtypes = [C.c_void_p, _dp, C.c_int32, _dp, _dp, _dp]
        lib.orc_step.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp,
                                 C.c_int, C.c_int64, C.c_uint64, C.c_int32, _dp, C.c_int, _ip, _dp]
        lib.orc_step.restype = C.c_int
        lib.orc_step_batch.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                       _dp, C.c_int, C.POINTER(C.c_int64), C.c_uint64, _ip, _ip,
                                       C.c_int, _dp]
        lib.orc_step_batch.restype = C.c_int
        _lib = lib
    return _lib


def _d(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """FP64 reference model built from a `ModelSpec` (paper_2601_22074_b300.inputs)."""

    def __init__(self, spec):
        lib = _load()
        self.spec = spec
        self._keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            self._keep.append(a)
            return a.ctypes.data_as({np.float64: _dp, np.int32: _ip, np.uint32: _up}[dt])

        o = spec.opt
        d = _Desc()
        d.nbody, d.njnt, d.nu, d.ngeom = spec.nbody, spec.njnt, spec.nu, spec.ngeom
        d.body_parent = arr(spec.body_parent, np.int32)
        for f in ("body_pos", "body_quat", "body_mass", "body_ipos", "body_inertia", "jnt_axis",
                  "jnt_pos", "jnt_armature", "jnt_reset_noise", "qpos_reset", "act_kp", "act_kd",
                  "geom_size", "geom_pos", "geom_quat", "geom_friction"):
            setattr(d, f, arr(getattr(spec, f), np.float64))
        for f in ("jnt_type", "jnt_body", "act_jnt", "geom_type", "geom_body"):
            setattr(d, f, arr(getattr(spec, f), np.int32))
        d.geom_contype = arr(spec.geom_contype, np.uint32)
        d.geom_conaffinity = arr(spec.geom_conaffinity, np.uint32)
        d.timestep = o.timestep
        d.gravity[:] = list(o.gravity)
        d.solref[:] = list(o.solref)
        d.solimp[:] = list(o.solimp)
        d.newton_iterations = o.newton_iterations
        d.newton_tolerance = o.newton_tolerance
        d.ls_iterations = o.ls_iterations
        d.pivot_tau = o.pivot_tau
        d.contact_cap = o.contact_cap
        d.push_period = o.push_period
        d.push_sigma = o.push_sigma
        if getattr(spec, "jnt_limited", None) is not None:
            d.jnt_limited = arr(spec.jnt_limited, np.int32)
            d.jnt_range = arr(spec.jnt_range, np.float64)
        if getattr(spec, "act_dcmotor", None) is not None:
            d.act_dcmotor = arr(spec.act_dcmotor, np.float64)
        if getattr(spec, "hfield_data", None) is not None:
            d.hfield_nrow, d.hfield_ncol = (int(x) for x in spec.hfield_data.shape)
            d.hfield_size[:] = [float(x) for x in spec.hfield_size]
            d.hfield_data = arr(spec.hfield_data, np.float64)
        err = C.create_string_buffer(256)
        h = lib.orc_model_create(C.byref(d), err, 256)
        if not h:
            raise ValueError("oracle model rejected: " + err.value.decode())
        self._h = h
        info = np.zeros(7, dtype=np.int32)
        lib.orc_model_info(h, info.ctypes.data_as(_ip))
        (self.nq, self.nv, self.nu, self.nbody, self.ngeom, self.npair,
         self.ncon_max) = (int(x) for x in info)
        self._lib = lib

    def __del__(self):
        try:
            self._lib.orc_model_destroy(self._h)
        except Exception:
            pass

    # ----------------------------------------------------------------- pieces
    def pairs(self) -> np.ndarray:
        out = np.zeros((max(self.npair, 1), 2), dtype=np.int32)
        self._lib.orc_model_pairs(self._h, out.ctypes.data_as(_ip))
        return out[: self.npair]

    @staticmethod
    def philox(ctr, key) -> np.ndarray:
        lib = _load()
        c = np.ascontiguousarray(ctr, dtype=np.uint32)
        k = np.ascontiguousarray(key, dtype=np.uint32)
        o = np.zeros(4, dtype=np.uint32)
        lib.orc_philox(c.ctypes.data_as(_up), k.ctypes.data_as(_up), o.ctypes.data_as(_up))
        return o

    def fk(self, qpos):
        q = _f64(qpos)
        nb, ng = self.nbody, self.ngeom
        out = dict(xpos=np.zeros((nb, 3)), xquat=np.zeros((nb, 4)), xmat=np.zeros((nb, 3, 3)),
                   xipos=np.zeros((nb, 3)), gxpos=np.zeros((ng, 3)), gxmat=np.zeros((ng, 3, 3)))
        self._lib.orc_fk(self._h, _d(q), *(_d(out[k]) for k in
                                           ("xpos", "xquat", "xmat", "xipos", "gxpos", "gxmat")))
        return out

    def mass_matrix(self, qpos, mass_scale=None) -> np.ndarray:
        M = np.zeros((self.nv, self.nv))
        ms = None if mass_scale is None else _f64(mass_scale)
        self._lib.orc_mass_matrix(self._h, _d(_f64(qpos)), _d(ms), _d(M))
        return M

    def rne(self, qpos, qvel, qacc, gravity=True, mass_scale=None) -> np.ndarray:
        tau = np.zeros(self.nv)
        ms = None if mass_scale is None else _f64(mass_scale)
        self._lib.orc_rne(self._h, _d(_f64(qpos)), _d(_f64(qvel)), _d(_f64(qacc)),
                          1 if gravity else 0, _d(ms), _d(tau))
        return tau

    def ltdl(self, M):
        L = np.zeros((self.nv, self.nv))
        D = np.zeros(self.nv)
        rc = self._lib.orc_ltdl(self._h, _d(_f64(M)), _d(L), _d(D))
        return L, D, rc

    def ltdl_solve(self, L, D, b) -> np.ndarray:
        x = _f64(b).copy()
        self._lib.orc_ltdl_solve(self._h, _d(_f64(L)), _d(_f64(D)), _d(x))
        return x

    def collide(self, qpos, cap=None) -> np.ndarray:
        cap = cap or max(self.ncon_max, 1)
        con = np.zeros((cap, CON_STRIDE))
        n = self._lib.orc_collide(self._h, _d(_f64(qpos)), _d(con), cap)
        return con[:n]

    def constraints(self, qpos, qvel, mass_scale=None, friction_scale=1.0):
        cap = max(self.ncon_max, 1)
        con = np.zeros((cap, CON_STRIDE))
        J = np.zeros((3 * cap, self.nv))
        aref = np.zeros(3 * cap)
        R = np.zeros(3 * cap)
        mu = np.zeros(cap)
        ms = None if mass_scale is None else _f64(mass_scale)
        nc = self._lib.orc_constraints(self._h, _d(_f64(qpos)), _d(_f64(qvel)), _d(ms),
                                       float(friction_scale), _d(con), cap, _d(J), _d(aref),
                                       _d(R), _d(mu))
        return dict(con=con[:nc], J=J[: 3 * nc], aref=aref[: 3 * nc], R=R[: 3 * nc],
                    mu=mu[:nc], nc=nc)

    @staticmethod
    def box_box(cA, RA, hA, cB, RB, hB, cap=8):
        lib = _load()
        con = np.zeros((cap, CON_STRIDE))
        axis = np.zeros(1, dtype=np.int32)
        minov = np.zeros(1)
        n = lib.orc_box_box(_d(_f64(cA)), _d(_f64(RA)), _d(_f64(hA)), _d(_f64(cB)), _d(_f64(RB)),
                            _d(_f64(hB)), _d(con), cap, axis.ctypes.data_as(_ip), _d(minov))
        return con[:n], int(axis[0]), float(minov[0])

    def limits(self, qpos, qvel, mass_scale=None):
        """Joint-limit rows of a state: dof, sign (+1 lower, -1 upper), dist, aref, R."""
        cap = max(self.spec.njnt, 1)
        dof = np.zeros(cap, dtype=np.int32)
        sg, dist, aref, R = (np.zeros(cap) for _ in range(4))
        ms = None if mass_scale is None else _f64(mass_scale)
        n = self._lib.orc_limits(self._h, _d(_f64(qpos)), _d(_f64(qvel)), _d(ms),
                                 dof.ctypes.data_as(_ip), _d(sg), _d(dist), _d(aref), _d(R), cap)
        return dict(dof=dof[:n], sign=sg[:n], dist=dist[:n], aref=aref[:n], R=R[:n], nl=n)

    @staticmethod
    def _limit_args(nv, Jl, arefl, Dl):
        if Jl is None or len(Dl) == 0:
            return 0, None, None, None
        return len(Dl), _d(_f64(Jl).reshape(-1)), _d(_f64(arefl)), _d(_f64(Dl))

    @staticmethod
    def cost(M, a_s, J, aref, D, mu, a, Jl=None, arefl=None, Dl=None) -> float:
        lib = _load()
        nv = M.shape[0]
        nc = len(mu)
        nl, jl, al, dl = Oracle._limit_args(nv, Jl, arefl, Dl)
        return lib.orc_cost(nv, _d(_f64(M)), _d(_f64(a_s)), nc, _d(_f64(J).reshape(-1)),
                            _d(_f64(aref)), _d(_f64(D)), _d(_f64(mu)), nl, jl, al, dl, _d(_f64(a)))

    @staticmethod
    def newton(M, a_s, J, aref, D, mu, a_init=None, maxiter=100, Jl=None, arefl=None, Dl=None):
        """Returns (qacc, contact forces [3nc], iterations), plus the limit forces [nl] when
        limit rows are given."""
        lib = _load()
        nv = M.shape[0]
        nc = len(mu)
        nl, jl, al, dl = Oracle._limit_args(nv, Jl, arefl, Dl)
        a = np.zeros(nv)
        f = np.zeros(max(3 * nc, 1))
        fl = np.zeros(max(nl, 1))
        ai = None if a_init is None else _f64(a_init)
        it = lib.orc_newton(nv, _d(_f64(M)), _d(_f64(a_s)), nc, _d(_f64(J).reshape(-1)),
                            _d(_f64(aref)), _d(_f64(D)), _d(_f64(mu)), nl, jl, al, dl, _d(ai),
                            _d(a), _d(f), _d(fl), maxiter)
        if Jl is None:
            return a, f[: 3 * nc], it
        return a, f[: 3 * nc], it, fl[:nl]

    def body_jacobian(self, qpos, body: int, point):
        """(Jp, Jr): [3, nv] point-velocity and angular-velocity Jacobians of body `body` at
        the world point `point`."""
        Jp = np.zeros((3, self.nv))
        Jr = np.zeros((3, self.nv))
        self._lib.orc_body_jacobian(self._h, _d(_f64(qpos)), int(body), _d(_f64(point)), _d(Jp), _d(Jr))
        return Jp, Jr

    def reset(self, seed: int, world: int):
        qpos = np.zeros(self.nq)
        qvel = np.zeros(self.nv)
        self._lib.orc_reset(self._h, C.c_uint64(seed), world, _d(qpos), _d(qvel))
        return qpos, qvel

    def step(self, qpos, qvel, qacc, ctrl, nsub=1, friction_scale=1.0, mass_scale=None,
             kp=None, kd=None, step_count=0, seed=0, world=0, want_contacts=False, body_inertia=None):
        """One env step (push event + nsub substeps). Returns new (qpos, qvel, qacc), stats,
        and the last substep's contacts (rows of CON_STRIDE) if asked."""
        qpos = _f64(qpos).copy()
        qvel = _f64(qvel).copy()
        qacc = _f64(qacc).copy()
        cap = max(self.ncon_max, 1)
        con = np.zeros((cap, CON_STRIDE)) if want_contacts else None
        stats = np.zeros(3, dtype=np.int32)
        ms = None if mass_scale is None else _f64(mass_scale)
        kpa = None if kp is None else _f64(kp)
        kda = None if kd is None else _f64(kd)
        ctrl_a = _f64(ctrl if ctrl is not None and len(ctrl) else np.zeros(max(self.nu, 1)))
        self._lib.orc_step(self._h, _d(qpos), _d(qvel), _d(qacc), _d(ctrl_a),
                           float(friction_scale), _d(ms), _d(kpa), _d(kda), int(nsub),
                           int(step_count), C.c_uint64(seed), int(world), _d(con), cap,
                           stats.ctypes.data_as(_ip),
                           None if body_inertia is None else _d(_f64(body_inertia)))
        out = dict(qpos=qpos, qvel=qvel, qacc=qacc, ncon=int(stats[0]), iters=int(stats[1]),
                   status=int(stats[2]))
        if want_contacts:
            out["contacts"] = con[: stats[0]]
        return out

    def step_batch(self, qpos, qvel, qacc, ctrl, nsub, params=None, step_count=None, seed=0,
                   world_id=None, nthreads=None):
        """Threaded FP64 env step over W worlds (in place on the float64 arrays)."""
        W = qpos.shape[0]
        nthreads = nthreads or os.cpu_count() or 1
        stats = np.zeros((W, 3), dtype=np.int32)
        sc = (np.zeros(W, dtype=np.int64) if step_count is None
              else np.ascontiguousarray(step_count, dtype=np.int64))
        wid = (None if world_id is None else np.ascontiguousarray(world_id, dtype=np.int32))
        fr = ms = kp = kd = bi = None
        if params is not None:
            fr, ms = _f64(params.friction_scale), _f64(params.mass_scale)
            kp, kd = _f64(params.kp), _f64(params.kd)
            if getattr(params, "inertia", None) is not None:
                bi = _f64(params.inertia)
        ctrl_a = _f64(ctrl) if self.nu else np.zeros((W, 1))
        self._lib.orc_step_batch(self._h, W, _d(qpos), _d(qvel), _d(qacc), _d(ctrl_a), _d(fr),
                                 _d(ms), _d(kp), _d(kd), int(nsub),
                                 sc.ctypes.data_as(C.POINTER(C.c_int64)), C.c_uint64(seed),
                                 None if wid is None else wid.ctypes.data_as(_ip),
                                 stats.ctypes.data_as(_ip), int(nthreads), _d(bi))
        return stats
