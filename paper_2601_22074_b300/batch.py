"""Python handle on the b3phys C ABI: models, batches, steps, readback.

Device memory and streams come from PyTorch (one uint8 tensor holds a whole
batch; calls run on torch's current stream); every step of the physics runs in
the library's CUDA kernels. Results land in caller-owned torch tensors, which
is how the paper's zero-copy TorchArray bridge (section "Software Design")
appears here.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence, Union

import numpy as np
import torch

from . import _lib as L
from .inputs import ModelSpec


def _stream_ptr(stream: Optional[torch.cuda.Stream] = None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Model:
    """A compiled model (host side). Keeps the descriptor arrays alive while created."""

    def __init__(self, spec: ModelSpec):
        lib = L.load()
        self.spec = spec
        keep = []

        def arr(x, dt, ptr):
            a = np.ascontiguousarray(x, dtype=dt)
            keep.append(a)
            return a.ctypes.data_as(ptr)

        d = L.ModelDesc()
        d.nbody, d.njnt, d.nu, d.ngeom = spec.nbody, spec.njnt, spec.nu, spec.ngeom
        dp, ip, up = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint32)
        d.body_parent = arr(spec.body_parent, np.int32, ip)
        for f in ("body_pos", "body_quat", "body_mass", "body_ipos", "body_inertia", "jnt_axis",
                  "jnt_pos", "jnt_armature", "jnt_reset_noise", "qpos_reset", "act_kp", "act_kd",
                  "geom_size", "geom_pos", "geom_quat", "geom_friction"):
            setattr(d, f, arr(getattr(spec, f), np.float64, dp))
        for f in ("jnt_type", "jnt_body", "act_jnt", "geom_type", "geom_body"):
            setattr(d, f, arr(getattr(spec, f), np.int32, ip))
        d.geom_contype = arr(spec.geom_contype, np.uint32, up)
        d.geom_conaffinity = arr(spec.geom_conaffinity, np.uint32, up)
        o = spec.opt
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
        if spec.jnt_limited is not None:
            d.jnt_limited = arr(spec.jnt_limited, np.int32, ip)
            d.jnt_range = arr(spec.jnt_range, np.float64, dp)
        if spec.act_dcmotor is not None:
            d.act_dcmotor = arr(spec.act_dcmotor, np.float64, dp)
        d.act_delay = int(spec.act_delay)
        if spec.hfield_data is not None:
            d.hfield_nrow, d.hfield_ncol = (int(x) for x in spec.hfield_data.shape)
            d.hfield_size[:] = [float(x) for x in spec.hfield_size]
            d.hfield_data = arr(spec.hfield_data, np.float64, dp)
        h = C.c_void_p()
        L.check(lib.b3p_model_create(C.byref(d), C.byref(h)), "b3p_model_create")
        self._h = h
        info = (C.c_int32 * 8)()
        L.check(lib.b3p_model_info(h, info), "b3p_model_info")
        (self.nq, self.nv, self.nu, self.nbody, self.ngeom, self.npair, self.ncon_max,
         self.nM) = (int(x) for x in info)

    def __del__(self):
        try:
            L.load().b3p_model_destroy(self._h)
        except Exception:
            pass


class Batch:
    """N worlds of one or more models in one device buffer."""

    def __init__(self, models: Union[Model, Sequence[Model]], nworld: Union[int, Sequence[int]],
                 write_contacts: bool = False, warps_per_block: int = 0, blocks_per_sm: int = 0,
                 schedule: int = 0, working_set: int = 0, history: int = 0, lane_solve: int = 0,
                 smem_scratch: int = 0, device: Union[str, torch.device] = "cuda"):
        lib = L.load()
        self.models: List[Model] = [models] if isinstance(models, Model) else list(models)
        self.nworld: List[int] = [nworld] if isinstance(nworld, int) else list(nworld)
        assert len(self.models) == len(self.nworld)
        self.device = torch.device(device)
        G = len(self.models)
        self._mh = (C.c_void_p * G)(*[m._h.value for m in self.models])
        self._nw = (C.c_int32 * G)(*self.nworld)
        self._opt = L.Options(warps_per_block, blocks_per_sm, 1 if write_contacts else 0, schedule,
                              working_set, history, lane_solve, smem_scratch)
        self.options = dict(warps_per_block=warps_per_block, blocks_per_sm=blocks_per_sm,
                            schedule=schedule, working_set=working_set, lane_solve=lane_solve)
        if smem_scratch:
            self.options["smem_scratch"] = smem_scratch
        self.history_depth = history
        sizes = L.Sizes()
        L.check(lib.b3p_batch_plan(self._mh, self._nw, G, C.byref(self._opt), C.byref(sizes)),
                "b3p_batch_plan")
        self.sizes = sizes
        self.buffer = torch.empty(int(sizes.total_bytes), dtype=torch.uint8, device=self.device)
        bufs = L.Buffers(self.buffer.data_ptr(), int(sizes.total_bytes))
        h = C.c_void_p()
        L.check(lib.b3p_batch_create(self._mh, self._nw, G, C.byref(self._opt), C.byref(bufs),
                                     _stream_ptr(), C.byref(h)), "b3p_batch_create")
        self._h = h
        self.write_contacts = write_contacts
        self.total_world = sum(self.nworld)
        self.world_start = list(np.cumsum([0] + self.nworld[:-1]))
        self._lib = lib

    def __del__(self):
        try:
            self._lib.b3p_batch_destroy(self._h)
        except Exception:
            pass

    # ---------------------------------------------------------------- helpers
    def _width(self, field: str) -> List[int]:
        if field == "qpos":
            return [m.nq for m in self.models]
        if field in ("qvel", "qacc"):
            return [m.nv for m in self.models]
        if field == "stats":
            return [4] * len(self.models)
        return [1] * len(self.models)

    def launch_info(self) -> dict:
        """The launch shape the batch settled on (b3p_batch_launch_info)."""
        out = (C.c_int32 * 5)()
        L.check(self._lib.b3p_batch_launch_info(self._h, out, 5), "b3p_batch_launch_info")
        return dict(warps_per_block=out[0], grid=out[1], smooth_smem_bytes=out[2], solve_smem_bytes=out[3],
                    lane_smem_bytes=out[4])

    def ctrl_size(self) -> int:
        return sum(m.nu * w for m, w in zip(self.models, self.nworld))

    # ---------------------------------------------------------------- calls
    def reset(self, seed: int, world_ids: Optional[torch.Tensor] = None,
              rng_ids: Optional[torch.Tensor] = None) -> None:
        n = 0 if world_ids is None else int(world_ids.numel())
        wp = None if world_ids is None else world_ids.data_ptr()
        rp = None if rng_ids is None else rng_ids.data_ptr()
        L.check(self._lib.b3p_reset(self._h, C.c_uint64(seed), wp, rp, n, _stream_ptr()),
                "b3p_reset")

    def set_param(self, group: int, field: str, values: torch.Tensor) -> None:
        v = values.to(device=self.device, dtype=torch.float32).contiguous()
        self._keep_param = v
        L.check(self._lib.b3p_set_world_param(self._h, group, L.PARAM[field], v.data_ptr(),
                                              _stream_ptr()), "b3p_set_world_param")

    def step(self, ctrl: Optional[torch.Tensor], decimation: int = 1) -> None:
        cp = None if ctrl is None else ctrl.data_ptr()
        L.check(self._lib.b3p_step(self._h, cp, decimation, _stream_ptr()), "b3p_step")

    def step_plain(self, ctrl: Optional[torch.Tensor], decimation: int = 1) -> None:
        """The per-stage, no-fusion comparator path (workspace allocated on first use)."""
        need = int(self._lib.b3p_plain_workspace_bytes(self._h))
        if getattr(self, "_plain_ws", None) is None or self._plain_ws.numel() < need:
            self._plain_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        cp = None if ctrl is None else ctrl.data_ptr()
        L.check(self._lib.b3p_step_plain(self._h, cp, decimation, self._plain_ws.data_ptr(), need,
                                         _stream_ptr()), "b3p_step_plain")

    def step_profile(self, ctrl: Optional[torch.Tensor], decimation: int = 1):
        """One staged step with per-stage kernel times (staged placement only); returns
        (ms per stage, launches per stage) as numpy arrays indexed like _lib.STAGES."""
        ms = (C.c_float * L.NSTAGES)()
        n = (C.c_int32 * L.NSTAGES)()
        cp = None if ctrl is None else ctrl.data_ptr()
        L.check(self._lib.b3p_step_profile(self._h, cp, decimation, ms, n, _stream_ptr()),
                "b3p_step_profile")
        return np.array(ms[:], dtype=np.float64), np.array(n[:], dtype=np.int64)

    def capture(self, ctrl_base: Optional[torch.Tensor], stride: int, decimation: int, nsteps: int,
                stream: torch.cuda.Stream) -> None:
        cp = None if ctrl_base is None else ctrl_base.data_ptr()
        L.check(self._lib.b3p_step_capture(self._h, cp, stride, decimation, nsteps,
                                           stream.cuda_stream), "b3p_step_capture")

    def replay(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        L.check(self._lib.b3p_graph_launch(self._h, _stream_ptr(stream)), "b3p_graph_launch")

    def get(self, field: str) -> torch.Tensor:
        dt = torch.float32 if field in ("qpos", "qvel", "qacc") else torch.int32
        n = sum(w * k for w, k in zip(self.nworld, self._width(field)))
        out = torch.empty(n, dtype=dt, device=self.device)
        L.check(self._lib.b3p_get_state(self._h, L.FIELD[field], out.data_ptr(), 4 * n,
                                        _stream_ptr()), "b3p_get_state")
        return out

    def set(self, field: str, values: torch.Tensor) -> None:
        dt = torch.float32 if field in ("qpos", "qvel", "qacc") else torch.int32
        v = values.to(device=self.device, dtype=dt).contiguous()
        L.check(self._lib.b3p_set_state(self._h, L.FIELD[field], v.data_ptr(), 4 * v.numel(),
                                        _stream_ptr()), "b3p_set_state")
        torch.cuda.current_stream().synchronize()

    def group_view(self, flat: torch.Tensor, field: str, group: int) -> torch.Tensor:
        widths = self._width(field)
        off = sum(w * k for w, k in zip(self.nworld[:group], widths[:group]))
        n = self.nworld[group] * widths[group]
        return flat[off:off + n].view(self.nworld[group], widths[group])

    def contacts(self):
        slots = sum(w * max(m.ncon_max, 1) for m, w in zip(self.models, self.nworld))
        out = torch.empty(slots * L.CON_FLOATS, dtype=torch.float32, device=self.device)
        cnt = torch.empty(self.total_world, dtype=torch.int32, device=self.device)
        L.check(self._lib.b3p_get_contacts(self._h, out.data_ptr(), 4 * out.numel(),
                                           cnt.data_ptr(), _stream_ptr()), "b3p_get_contacts")
        return out.view(slots, L.CON_FLOATS), cnt

    def diffik(self, group: int, body: int, offset, target_pos: torch.Tensor, ctrl: torch.Tensor,
               target_quat: Optional[torch.Tensor] = None, damping: float = 0.05) -> None:
        """Damped-least-squares IK targets for the group's actuators, written into ctrl
        (the flat targets of the whole batch)."""
        off = (C.c_float * 3)(*[float(x) for x in offset])
        tp = target_pos.to(device=self.device, dtype=torch.float32).contiguous()
        tq = None if target_quat is None else target_quat.to(device=self.device, dtype=torch.float32).contiguous()
        self._keep_ik = (tp, tq)
        L.check(self._lib.b3p_diffik(self._h, group, body, off, tp.data_ptr(),
                                     None if tq is None else tq.data_ptr(), float(damping), ctrl.data_ptr(),
                                     _stream_ptr()), "b3p_diffik")

    def raycast(self, group: int, body: int, origins: torch.Tensor, directions: torch.Tensor,
                max_dist: float = 10.0, world_only: bool = True) -> torch.Tensor:
        """Distances [W_g, nray] along rays fixed to `body` (body-frame origins and unit
        directions [nray, 3])."""
        o = origins.to(device=self.device, dtype=torch.float32).contiguous()
        d = directions.to(device=self.device, dtype=torch.float32).contiguous()
        n = int(o.shape[0])
        out = torch.empty((self.nworld[group], n), dtype=torch.float32, device=self.device)
        L.check(self._lib.b3p_raycast(self._h, group, body, n, o.data_ptr(), d.data_ptr(), float(max_dist),
                                      1 if world_only else 0, out.data_ptr(), _stream_ptr()), "b3p_raycast")
        return out

    def raycast_hits(self, group: int, body: int, origins: torch.Tensor, directions: torch.Tensor,
                     max_dist: float = 10.0, world_only: bool = True, hierarchy: bool = True):
        """(distances [W_g, nray], hit positions [W_g, nray, 3], normals [W_g, nray, 3]);
        hierarchy=False tests every geom in turn (the reference for the hierarchy)."""
        o = origins.to(device=self.device, dtype=torch.float32).contiguous()
        d = directions.to(device=self.device, dtype=torch.float32).contiguous()
        n, W = int(o.shape[0]), self.nworld[group]
        dist = torch.empty((W, n), dtype=torch.float32, device=self.device)
        pos = torch.empty((W, n, 3), dtype=torch.float32, device=self.device)
        nrm = torch.empty((W, n, 3), dtype=torch.float32, device=self.device)
        flags = (1 if world_only else 0) | (0 if hierarchy else 2)
        L.check(self._lib.b3p_raycast_hits(self._h, group, body, n, o.data_ptr(), d.data_ptr(), float(max_dist),
                                           flags, dist.data_ptr(), pos.data_ptr(), nrm.data_ptr(), _stream_ptr()),
                "b3p_raycast_hits")
        return dist, pos, nrm

    def history(self, group: int, world: int):
        """(states [n, nq + nv] oldest first, n) of one world's ring of recent states."""
        m = self.models[group]
        dst = torch.empty((self.history_depth, m.nq + m.nv), dtype=torch.float32, device=self.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=self.device)
        L.check(self._lib.b3p_get_history(self._h, group, world, dst.data_ptr(), cnt.data_ptr(), _stream_ptr()),
                "b3p_get_history")
        n = int(cnt.item())
        return dst[:n], n

    def observe(self, group: int, ctrl: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Velocity-task observation terms of one group, [W_g, width] on the device
        (ctrl: the flat targets of the whole batch, as passed to step)."""
        width = int(self._lib.b3p_observe_width(self._h, group))
        if width < 0:
            raise ValueError(f"no group {group}")
        out = torch.empty((self.nworld[group], width), dtype=torch.float32, device=self.device)
        cp = None if ctrl is None else ctrl.data_ptr()
        L.check(self._lib.b3p_observe(self._h, group, cp, out.data_ptr(), _stream_ptr()), "b3p_observe")
        return out

    def contact_sensor(self, group: int, bodies: torch.Tensor, state: torch.Tensor, threshold: float = 1.0,
                       dt: float = 0.0, history: Optional[torch.Tensor] = None,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Net contact force [W_g, n, 3] on the listed bodies; advances the caller's air-time
        state [W_g, n, 4] (in contact, air time, contact time, last air time) by dt. With
        `history` [W_g, n, depth, 3] the force also goes into slot (step count - 1) mod depth
        of each world's ring. `out` (optional) receives the forces in place."""
        ids = bodies.to(device=self.device, dtype=torch.int32).contiguous()
        self._keep_sensor = ids
        n = int(ids.numel())
        assert state.shape == (self.nworld[group], n, 4) and state.dtype == torch.float32
        force = out if out is not None else torch.empty((self.nworld[group], n, 3), dtype=torch.float32,
                                                        device=self.device)
        if history is None:
            L.check(self._lib.b3p_contact_sensor(self._h, group, ids.data_ptr(), n, float(threshold), float(dt),
                                                 state.data_ptr(), force.data_ptr(), _stream_ptr()),
                    "b3p_contact_sensor")
        else:
            assert history.shape[:2] == (self.nworld[group], n) and history.shape[3] == 3
            L.check(self._lib.b3p_contact_sensor_history(self._h, group, ids.data_ptr(), n, float(threshold),
                                                         float(dt), state.data_ptr(), force.data_ptr(),
                                                         history.data_ptr(), int(history.shape[2]),
                                                         _stream_ptr()), "b3p_contact_sensor_history")
        return force

    def reward(self, group: int, cfg: "RewardConfig", cmd: torch.Tensor, action: Optional[torch.Tensor],
               prev_action: Optional[torch.Tensor], sensor_state: Optional[torch.Tensor], out: dict) -> None:
        """Reward and termination of the velocity-tracking task for one group (b3p_reward), into
        the caller's tensors out["reward"] [W_g], out["terms"] [W_g, 10], out["episode"]
        [W_g, 10] (accumulated) and out["done"] [W_g] (int32 bits)."""
        c = cfg.c_struct()
        self._keep_reward = (c, cfg)
        ap = None if action is None else action.data_ptr()
        pp = None if prev_action is None else prev_action.data_ptr()
        sp = None if sensor_state is None else sensor_state.data_ptr()
        L.check(self._lib.b3p_reward(self._h, group, C.byref(c), cmd.data_ptr(), ap, pp, sp,
                                     out["reward"].data_ptr(), out["terms"].data_ptr(), out["episode"].data_ptr(),
                                     out["done"].data_ptr(), _stream_ptr()), "b3p_reward")

    def state_bytes(self) -> int:
        return int(self._lib.b3p_state_bytes(self._h))

    def state_save(self) -> torch.Tensor:
        out = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        L.check(self._lib.b3p_state_save(self._h, out.data_ptr(), out.numel(), _stream_ptr()),
                "b3p_state_save")
        return out

    def state_restore(self, snap: torch.Tensor) -> None:
        L.check(self._lib.b3p_state_restore(self._h, snap.data_ptr(), snap.numel(),
                                            _stream_ptr()), "b3p_state_restore")


def fp32_peak(reps: int = 5):
    """(FLOP/s, SM count): the current device's measured FP32 FMA throughput
    (b3p_fp32_peak), the ALU roof of the step's roofline."""
    fl = C.c_double()
    sms = C.c_int32()
    L.check(L.load().b3p_fp32_peak(int(reps), C.byref(fl), C.byref(sms), _stream_ptr()), "b3p_fp32_peak")
    return float(fl.value), int(sms.value)


class RewardConfig:
    """Weights and thresholds of b3p_reward (terms in _lib.REWARD_TERMS order)."""

    def __init__(self, weight, dt: float, sigma_lin: float = 0.5, sigma_ang: float = 0.5,
                 air_time_target: float = 0.4, min_base_height: float = 0.0, max_tilt: float = 0.0,
                 max_episode_steps: int = 0, feet=(), illegal=()):
        assert len(weight) == L.REWARD_NTERMS
        self.weight = [float(w) for w in weight]
        self.dt, self.sigma_lin, self.sigma_ang = float(dt), float(sigma_lin), float(sigma_ang)
        self.air_time_target = float(air_time_target)
        self.min_base_height, self.max_tilt = float(min_base_height), float(max_tilt)
        self.max_episode_steps = int(max_episode_steps)
        self.feet = np.ascontiguousarray(feet, dtype=np.int32)
        self.illegal = np.ascontiguousarray(illegal, dtype=np.int32)

    def c_struct(self) -> L.RewardCfg:
        c = L.RewardCfg()
        c.weight[:] = self.weight
        c.sigma_lin, c.sigma_ang, c.air_time_target = self.sigma_lin, self.sigma_ang, self.air_time_target
        c.dt, c.min_base_height, c.max_tilt = self.dt, self.min_base_height, self.max_tilt
        c.max_episode_steps = self.max_episode_steps
        c.nfeet, c.nillegal = len(self.feet), len(self.illegal)
        ip = C.POINTER(C.c_int32)
        c.feet_host = self.feet.ctypes.data_as(ip) if len(self.feet) else None
        c.illegal_host = self.illegal.ctypes.data_as(ip) if len(self.illegal) else None
        return c
