"""The C-ABI library loads and exports every symbol include/diffsim.h
declares; host-side validation rejects bad configurations before touching a
GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2509_10247_b300 import binding, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def declared_functions(header="diffsim.h", prefix="sim_"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(%s[a-z0-9_]+)\s*\(" % prefix, src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.SYMBOLS) == names


def test_header_config_layout_matches_binding():
    # sizeof(sim_config) from the header's field list: 4-byte fields only
    src = open(os.path.join(ROOT, "include", "diffsim.h")).read()
    body = src[src.index("typedef struct sim_config {"):src.index("} sim_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    n = 0
    for decl in re.findall(r"(?:int32_t|float)\s+([^;]+);", body):
        for item in decl.split(","):
            m = re.search(r"\[(\d+)\]", item)
            n += int(m.group(1)) if m else 1
    assert ctypes.sizeof(binding.SimConfig) == 4 * n


def test_version_and_errors(lib):
    assert "sm_103a" in binding.sim_version()
    assert binding.sim_strerror(0) == "ok"
    assert binding.sim_strerror(-2) == "null pointer"
    assert binding.sim_strerror(5) == "unknown error"
    assert binding.sim_state_dim(0) == 12 and binding.sim_state_dim(1) == 13
    assert binding.sim_action_dim(0) == 3 and binding.sim_action_dim(1) == 4
    assert binding.sim_state_dim(2) == 12 and binding.sim_action_dim(2) == 3
    assert binding.sim_state_dim(3) == 15 and binding.sim_action_dim(3) == 4
    assert binding.sim_state_dim(9) == -1


def _create_rc(lib, cfg):
    h = ctypes.c_void_p()
    rc = lib.sim_create(ctypes.byref(cfg), ctypes.byref(h))
    return rc, h.value


@pytest.mark.parametrize("field,value,code", [
    ("model", 5, -1), ("n_env", 0, -3), ("n_agent", 0, -3), ("n_agent", 33, -3), ("horizon", 0, -3),
    ("dt", 0.0, -1), ("dt", float("nan"), -1), ("ema_alpha", 1.5, -1), ("cam_h", 0, -3),
    ("cam_hfov", 0.0, -1), ("cam_range", -1.0, -1), ("pool_size", -1, -3), ("terminate", 2, -1),
    ("tape_hits", 3, -1), ("cull", 3, -1), ("warps_per_cta", 9, -1), ("rays_per_thread", 7, -1),
    ("ctas_per_sm", -1, -1),
])
def test_create_rejects_bad_config(lib, field, value, code):
    cfg = binding.make_config(synth.preset("pointmass_64env_depth16x9_10sph"))
    setattr(cfg, field, value)
    rc, h = _create_rc(lib, cfg)
    assert rc == code and h is None


def test_create_rejects_bad_cast_mode_and_rigid_params(lib):
    cfg = binding.make_config(synth.preset("pointmass_64env_depth16x9_10sph"))
    cfg.cast_mode = 2
    assert _create_rc(lib, cfg)[0] == -1
    cfg = binding.make_config(synth.preset("pointmass_64env_depth16x9_10sph"))
    cfg.task = 2
    assert _create_rc(lib, cfg)[0] == -1
    cfg = binding.make_config(synth.preset("pointmass_64env_depth16x9_10sph"))
    cfg.imu_walk[1] = -0.1
    assert _create_rc(lib, cfg)[0] == -1
    cfg = binding.make_config(synth.preset("rigid_4096env_depth64x48_40sph20box"))
    cfg.inertia[1] = 0.0
    assert _create_rc(lib, cfg)[0] == -1
    cfg = binding.make_config(synth.preset("rigid_65536env_256obst_depth_lidar"))
    cfg.lid_elev_lo, cfg.lid_elev_hi = 0.5, 0.1
    assert _create_rc(lib, cfg)[0] == -1


def test_null_pointers(lib):
    cfg = binding.make_config(synth.preset("pointmass_64env_depth16x9_10sph"))
    assert lib.sim_create(None, None) == -2
    assert lib.sim_create(ctypes.byref(cfg), None) == -2
    assert lib.sim_destroy(None) == 0
    assert lib.sim_rollout(None, None, None, None, None, None, None, None) == -2
    assert lib.sim_backward(None, None, None, None, None, None, None, None) == -2
    assert lib.sim_set_scene(None, None, None, None, None, 0, None, None) == -2
    assert lib.sim_set_scene_ex(None, None) == -2
    assert lib.sim_rollout_ex(None, None, None) == -2
    assert lib.sim_step_ex(None, None, None) == -2
    assert lib.sim_backward_ex(None, None, None) == -2
    assert lib.sim_get_gate_index(None, None, None) == -2
    assert lib.sim_set_gate_index(None, None, None) == -2
    assert lib.sim_last_status(None, None, None) == -2
    assert lib.sim_render_taped(None, None, None, None, None, None) == -2
    assert lib.sim_render_hits(None, None, None, None, None, None) == -2
    assert lib.sim_step_backward_taped(None, None, None, None, None, None, None, None, None, None, None, None,
                                       None) == -2


def test_valid_config_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = binding.make_config(synth.preset("pointmass_64env_depth16x9_10sph"))
    rc, h = _create_rc(lib, cfg)
    assert rc == -4 and h is None


def test_graph_and_profiling_null_pointers(lib):
    assert lib.sim_profile(None, 1) == -2
    assert lib.sim_kernel_times(None, None, None, 0) == -2
    assert lib.sim_graph_create(None, None, None) == -2
    assert lib.sim_graph_launch(None, None) == -2
    assert lib.sim_graph_kernels(None, None) == -2
    assert lib.sim_graph_destroy(None) == 0


def test_rollout_io_layout_matches_header():
    src = open(os.path.join(ROOT, "include", "diffsim.h")).read()
    body = src[src.index("typedef struct sim_rollout_io {"):src.index("} sim_rollout_io;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    n = sum(len(d.split(",")) for d in re.findall(r"\*\s*([^;]+);", body))
    assert ctypes.sizeof(binding.SimRolloutIO) == 8 * n
    assert [f for f, _ in binding.SimRolloutIO._fields_][-2:] == ["hits_cam", "hits_lidar"]


def test_graph_io_layout_matches_header():
    src = open(os.path.join(ROOT, "include", "diffsim.h")).read()
    body = src[src.index("typedef struct sim_graph_io {"):src.index("} sim_graph_io;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    n = sum(len(d.split(",")) for d in re.findall(r"\*\s*([^;]+);", body))
    assert ctypes.sizeof(binding.SimGraphIO) == 8 * n


def test_surrogate_symbols_exported(lib):
    from paper_2509_10247_b300 import surrogate
    names = declared_functions("surrogate.h", "surr_")
    assert sorted(surrogate.SYMBOLS) == names
    for n in names:
        assert hasattr(lib, n), n
    src = open(os.path.join(ROOT, "include", "surrogate.h")).read()
    assert "#define SURR_NPARAM %d" % surrogate.NPARAM in src
    assert "#define SURR_NSTATS %d" % surrogate.NSTATS in src
    assert sum(n for _, n in surrogate.STATS_LAYOUT) == surrogate.NSTATS
    from paper_2509_10247_b300 import synth
    assert sum(int(np.prod(s)) for _, s in synth.SURR_SHAPES) == surrogate.NPARAM


def test_surrogate_rejects_bad_config(lib):
    from paper_2509_10247_b300 import surrogate, synth
    phys = binding.make_config(synth.preset("surrogate_rigid_65536env_32step"))
    for kw in (dict(batch=100), dict(batch=0), dict(lr=0.0), dict(beta1=1.0), dict(margin=-1.0)):
        cfg = surrogate.SurrConfig(batch=kw.get("batch", 256), splits=0, lr=kw.get("lr", 1e-3),
                                   beta1=kw.get("beta1", 0.9), beta2=0.999, eps=1e-8, margin=kw.get("margin", 0.1))
        h = ctypes.c_void_p()
        assert lib.surr_create(ctypes.byref(cfg), ctypes.byref(phys), ctypes.byref(h)) in (-1, -3)
    cfg = surrogate.SurrConfig(batch=256, splits=0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, margin=0.1)
    pm = binding.make_config(synth.preset("pointmass_64env_depth16x9_10sph"))
    h = ctypes.c_void_p()
    assert lib.surr_create(ctypes.byref(cfg), ctypes.byref(pm), ctypes.byref(h)) == -9
    assert lib.surr_create(None, None, None) == -2
    assert lib.surr_destroy(None) == 0
    assert lib.surr_rollout(None, None, None, 0, 0, None, None, None, None) == -2


def test_policy_symbols_exported(lib):
    from paper_2509_10247_b300 import policy
    names = declared_functions("policy.h", "pol_")
    assert sorted(policy.SYMBOLS) == names
    for n in names:
        assert hasattr(lib, n), n
    L = policy._lib()
    h = ctypes.c_void_p()
    assert L.pol_create(0, 0, 1.0, 0, 1.0, ctypes.byref(h)) == -3
    assert L.pol_create(4, 10, 0.0, 0, 1.0, ctypes.byref(h)) == -1
    assert L.pol_create(4, 10, 1.0, 0, 1.0, None) == -2
    assert L.pol_destroy(None) == 0
    assert L.pol_backward(None, None, None, None, None, None) == -2
