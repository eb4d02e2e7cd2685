"""ctypes declarations of the b3phys C ABI (include/b3phys.h). Marshalling only.

Loading fails loudly when the compiled library is missing: there is no CPU or
Python fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libb3phys.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint32)
_vp = C.c_void_p

OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "BAD_MODEL", -3: "WORKSPACE_TOO_SMALL", -4: "CUDA",
          -5: "GRAPH_STALE", -6: "TIMEOUT", -7: "BUSY", -8: "UNSUPPORTED"}
FIELD = {"qpos": 0, "qvel": 1, "qacc": 2, "status": 3, "stats": 4, "step_count": 5}
PARAM = {"friction_scale": 0, "mass_scale": 1, "kp": 2, "kd": 3, "body_inertia": 4}
CON_FLOATS = 24
STATIC_SCRATCH_DOUBLES = 4194304   # B3P_STATIC_SCRATCH_DOUBLES of include/b3phys.h
STATUS_NAN, STATUS_OVERFLOW, STATUS_NOT_CONVERGED, STATUS_FP64, STATUS_BAD_PIVOT, STATUS_IDLE = (
    1, 2, 4, 8, 16, 32)


class ModelDesc(C.Structure):
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
        ("jnt_limited", _ip), ("jnt_range", _dp), ("act_dcmotor", _dp), ("act_delay", C.c_int32),
        ("hfield_nrow", C.c_int32), ("hfield_ncol", C.c_int32), ("hfield_size", C.c_double * 2),
        ("hfield_data", _dp),
    ]


REWARD_NTERMS, REWARD_MAXBODIES = 10, 16
REWARD_TERMS = ("track_lin_vel", "track_ang_vel", "lin_vel_z", "ang_vel_xy", "action_rate", "joint_limit",
                "feet_slip", "feet_air_time", "upright", "joint_acc")
DONE_TERMINATED, DONE_TIMEOUT, DONE_NONFINITE, DONE_LOW, DONE_TILT, DONE_ILLEGAL = 1, 2, 4, 8, 16, 32


class RewardCfg(C.Structure):
    _fields_ = [("weight", C.c_float * REWARD_NTERMS), ("sigma_lin", C.c_float), ("sigma_ang", C.c_float),
                ("air_time_target", C.c_float), ("dt", C.c_float), ("min_base_height", C.c_float),
                ("max_tilt", C.c_float), ("max_episode_steps", C.c_int32), ("nfeet", C.c_int32),
                ("feet_host", _ip), ("nillegal", C.c_int32), ("illegal_host", _ip)]


class Options(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("write_contacts", C.c_int32), ("schedule", C.c_int32),
                ("working_set", C.c_int32), ("history", C.c_int32), ("lane_solve", C.c_int32),
                ("smem_scratch", C.c_int32)]


class Sizes(C.Structure):
    _fields_ = [("total_bytes", C.c_uint64), ("model_bytes", C.c_uint64),
                ("state_bytes", C.c_uint64), ("param_bytes", C.c_uint64),
                ("contact_bytes", C.c_uint64), ("scratch_bytes", C.c_uint64),
                ("nworld", C.c_int32), ("smem_bytes_per_world", C.c_int32)]


class Buffers(C.Structure):
    _fields_ = [("base", _vp), ("bytes", C.c_uint64)]


class ServerCfg(C.Structure):
    _fields_ = [("nmodels", C.c_int32), ("models", C.POINTER(_vp)), ("hbm_budget_bytes", C.c_double),
                ("max_worlds_per_model", C.c_int32), ("decimation", C.c_int32),
                ("sigma_host", C.POINTER(C.c_float)), ("options", Options),
                ("max_inflight_ticks", C.c_int32), ("run_thread", C.c_int32), ("device", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("model", C.c_int32), ("nworld", C.c_int32), ("horizon", C.c_int32),
                ("seed", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("id", C.c_int64), ("model", C.c_int32), ("nworld", C.c_int32),
                ("qpos", C.POINTER(C.c_float)), ("qvel", C.POINTER(C.c_float)),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("ticks", C.c_int64), ("world_steps", C.c_int64), ("submitted", C.c_int64),
                ("completed", C.c_int64), ("queued", C.c_int32), ("active", C.c_int32),
                ("pending", C.c_int32), ("reserved", C.c_int32)]


# (name, restype, argtypes)
NSTAGES = 8
STAGES = ("load", "kinematics", "bias", "mass", "collide", "solve", "integrate", "store")

SIGNATURES = [
    ("b3p_last_error", C.c_char_p, []),
    ("b3p_version", C.c_char_p, []),
    ("b3p_model_create", C.c_int32, [C.POINTER(ModelDesc), C.POINTER(_vp)]),
    ("b3p_model_destroy", None, [_vp]),
    ("b3p_model_info", C.c_int32, [_vp, _ip]),
    ("b3p_batch_plan", C.c_int32, [C.POINTER(_vp), _ip, C.c_int32, C.POINTER(Options),
                                   C.POINTER(Sizes)]),
    ("b3p_batch_create", C.c_int32, [C.POINTER(_vp), _ip, C.c_int32, C.POINTER(Options),
                                     C.POINTER(Buffers), _vp, C.POINTER(_vp)]),
    ("b3p_batch_destroy", None, [_vp]),
    ("b3p_batch_info", C.c_int32, [_vp, _ip, C.c_int32]),
    ("b3p_batch_launch_info", C.c_int32, [_vp, _ip, C.c_int32]),
    ("b3p_reset", C.c_int32, [_vp, C.c_uint64, _vp, _vp, C.c_int32, _vp]),
    ("b3p_set_world_param", C.c_int32, [_vp, C.c_int32, C.c_int32, _vp, _vp]),
    ("b3p_step", C.c_int32, [_vp, _vp, C.c_int32, _vp]),
    ("b3p_step_static_scratch", C.c_int32, [_vp, _vp, C.c_int32, _vp]),
    ("b3p_step_capture", C.c_int32, [_vp, _vp, C.c_int64, C.c_int32, C.c_int32, _vp]),
    ("b3p_graph_launch", C.c_int32, [_vp, _vp]),
    ("b3p_get_state", C.c_int32, [_vp, C.c_int32, _vp, C.c_size_t, _vp]),
    ("b3p_set_state", C.c_int32, [_vp, C.c_int32, _vp, C.c_size_t, _vp]),
    ("b3p_get_contacts", C.c_int32, [_vp, _vp, C.c_size_t, _vp, _vp]),
    ("b3p_plain_workspace_bytes", C.c_size_t, [_vp]),
    ("b3p_step_plain", C.c_int32, [_vp, _vp, C.c_int32, _vp, C.c_size_t, _vp]),
    ("b3p_step_profile", C.c_int32, [_vp, _vp, C.c_int32, C.POINTER(C.c_float), _ip, _vp]),
    ("b3p_fp32_peak", C.c_int32, [C.c_int32, _dp, _ip, _vp]),
    ("b3p_server_create", C.c_int32, [C.POINTER(ServerCfg), C.POINTER(_vp)]),
    ("b3p_server_destroy", None, [_vp]),
    ("b3p_server_capacity", C.c_int32, [_vp, _ip, C.c_int32]),
    ("b3p_server_submit", C.c_int32, [_vp, C.POINTER(Request), C.POINTER(C.c_int64)]),
    ("b3p_server_tick", C.c_int32, [_vp, _ip]),
    ("b3p_server_poll", C.c_int32, [_vp, C.POINTER(Result), C.c_int32, _ip]),
    ("b3p_server_release", C.c_int32, [_vp, C.c_int64]),
    ("b3p_server_get_stats", C.c_int32, [_vp, C.POINTER(ServerStats)]),
    ("b3p_server_now", C.c_double, [_vp]),
    ("b3p_diffik", C.c_int32, [_vp, C.c_int32, C.c_int32, C.POINTER(C.c_float), _vp, _vp, C.c_float, _vp, _vp]),
    ("b3p_raycast", C.c_int32, [_vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp, C.c_float, C.c_int32, _vp, _vp]),
    ("b3p_raycast_hits", C.c_int32, [_vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp, C.c_float, C.c_int32, _vp,
                                     _vp, _vp, _vp]),
    ("b3p_get_history", C.c_int32, [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp]),
    ("b3p_observe_width", C.c_int32, [_vp, C.c_int32]),
    ("b3p_observe", C.c_int32, [_vp, C.c_int32, _vp, _vp, _vp]),
    ("b3p_contact_sensor", C.c_int32, [_vp, C.c_int32, _vp, C.c_int32, C.c_float, C.c_float, _vp, _vp, _vp]),
    ("b3p_contact_sensor_history", C.c_int32, [_vp, C.c_int32, _vp, C.c_int32, C.c_float, C.c_float, _vp, _vp,
                                               _vp, C.c_int32, _vp]),
    ("b3p_reward", C.c_int32, [_vp, C.c_int32, C.POINTER(RewardCfg), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("b3p_set_idle", C.c_int32, [_vp, _vp, C.c_int32, C.c_int32, _vp]),
    ("b3p_sample_targets", C.c_int32, [_vp, _vp, _vp, _vp]),
    ("b3p_gather_state", C.c_int32, [_vp, C.c_int32, C.c_int32, _vp, C.c_int32, _vp, _vp]),
    ("b3p_state_bytes", C.c_size_t, [_vp]),
    ("b3p_state_save", C.c_int32, [_vp, _vp, C.c_size_t, _vp]),
    ("b3p_state_restore", C.c_int32, [_vp, _vp, C.c_size_t, _vp]),
]

_lib = None


def load():
    """Load libb3phys.so (built by paper_2601_22074_b300.build); raise if absent.
    B3P_LIB_PATH selects another build of the same sources (the tracing variant)."""
    global _lib
    if _lib is None:
        path = os.environ.get("B3P_LIB_PATH", LIB_PATH)
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run paper_2601_22074_b300.build.build() "
                              "(there is no fallback path)")
        lib = C.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class B3PError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().b3p_last_error().decode()
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str) -> None:
    if code != OK:
        raise B3PError(code, where)
