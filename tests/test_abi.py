"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/b3phys.h declares, compiles the models into the same structure the
oracle derives independently, rejects malformed descriptors, and plans batch sizes."""
import os
import re

import numpy as np
import pytest

from oracle import Oracle
from paper_2601_22074_b300 import _lib as L
from paper_2601_22074_b300 import build, inputs as I
from paper_2601_22074_b300.batch import Model

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "b3phys.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(b3p_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = L.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in L.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


@pytest.mark.parametrize("name", ["pendulum", "quadruped", "humanoid", "spatial_chain"])
def test_model_structure_matches_oracle(name):
    spec = getattr(I, name)() if name != "pendulum" else I.pendulum(3)
    m, o = Model(spec), Oracle(spec)
    assert (m.nq, m.nv, m.nu, m.nbody, m.ngeom, m.npair, m.ncon_max) == \
           (o.nq, o.nv, o.nu, o.nbody, o.ngeom, o.npair, o.ncon_max)
    if name == "humanoid":
        assert m.nM == 341


def _broken(**kw):
    spec = I.quadruped()
    for k, v in kw.items():
        arr = getattr(spec, k).copy()
        idx, val = v
        arr[idx] = val
        setattr(spec, k, arr)
    return spec


@pytest.mark.parametrize("kw,code", [
    (dict(body_parent=(3, 5)), "BAD_MODEL"),            # parent after child
    (dict(jnt_body=(0, 2)), "BAD_MODEL"),               # free joint moved off a world child
    (dict(act_jnt=(0, 0)), "BAD_MODEL"),                 # actuator on the free joint
    (dict(act_jnt=(1, 1)), "BAD_MODEL"),                 # two actuators on one joint
    (dict(jnt_axis=(1, [0, 0, 0])), "BAD_MODEL"),        # zero hinge axis
    (dict(geom_type=(3, 1)), "OK"),                      # sphere on a thigh is still plane-paired
])
def test_model_rejects_malformed_descriptors(kw, code):
    spec = _broken(**kw)
    if code == "OK":
        Model(spec)
        return
    with pytest.raises(L.B3PError) as e:
        Model(spec)
    assert L.ERRORS[e.value.code] == code


def test_unsupported_pair_is_reported():
    spec = I.quadruped()
    ct = spec.geom_contype.copy()
    ca = spec.geom_conaffinity.copy()
    ca[:] = 3   # robot geoms now collide with each other: sphere-capsule etc.
    spec.geom_conaffinity = ca
    spec.geom_contype = ct
    with pytest.raises(L.B3PError) as e:
        Model(spec)
    assert L.ERRORS[e.value.code] == "UNSUPPORTED"


def test_batch_plan_scales_with_worlds():
    import ctypes as C
    lib = L.load()
    m = Model(I.humanoid())
    sizes = []
    for W in (1024, 8192):
        mh = (C.c_void_p * 1)(m._h.value)
        nw = (C.c_int32 * 1)(W)
        s = L.Sizes()
        L.check(lib.b3p_batch_plan(mh, nw, 1, None, C.byref(s)), "plan")
        sizes.append(s)
    a, b = sizes
    assert b.state_bytes > 7 * a.state_bytes
    assert b.total_bytes < 256 << 20            # 8192 humanoids fit in well under 256 MB
    assert a.smem_bytes_per_world == b.smem_bytes_per_world
    assert a.smem_bytes_per_world < 24 << 10    # fits several worlds per SM


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2601_22074_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), f
                assert "liboracle" not in src and "oracle.h" not in src, f


def test_invalid_limit_and_motor_descriptors_are_refused():
    import dataclasses
    from paper_2601_22074_b300.batch import Model
    spec = I.with_limits(I.pendulum(2), 0.5)
    bad = dataclasses.replace(spec, jnt_range=spec.jnt_range[:, ::-1].copy())
    with pytest.raises(RuntimeError, match="BAD_MODEL"):
        Model(bad)
    q = I.with_dcmotor(I.quadruped(), 10.0, 0.0, 5.0)
    with pytest.raises(RuntimeError, match="BAD_MODEL"):
        Model(q)
    with pytest.raises(RuntimeError, match="BAD_MODEL"):
        Model(I.with_delay(I.quadruped(), 65))
