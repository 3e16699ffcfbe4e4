"""Host logic of the launch-shape autotuner: key, selection, parity gate,
cache (no GPU: the measurement is replaced by a fake runner)."""
import json

import pytest

from paper_2509_10247_b300 import autotune, synth


def _wl():
    p = synth.preset("swarm_16384env_8agent_8maps_depth16x9", n_env=16, horizon=4)
    return p, synth.make_inputs(p, seed=0)


def test_key_ignores_name_and_exec_fields_but_not_physics():
    p, inp = _wl()
    k = autotune.workload_key(p, inp)
    assert autotune.workload_key(dict(p, name="other"), inp) == k
    assert autotune.workload_key(dict(p, dt=0.02), inp) != k
    q = synth.preset("swarm_16384env_8agent_8maps_depth16x9", n_env=16, horizon=4,
                     map_counts=[(1, 1)] * 8)
    assert autotune.workload_key(q, synth.make_inputs(q, seed=0)) != k


def test_selection_admits_only_bitwise_equal_candidates(tmp_path):
    p, inp = _wl()
    ref = [1, 2, 3]
    table = {1: (5.0, ref), 2: (1.0, [1, 2, 4]), 3: (2.0, ref), 4: (None, None), 5: (3.0, ref)}

    def runner(ex):
        r = ex["rays_per_thread"]
        return (9.0, ref) if r == 0 else table[r]

    cands = [dict(rays_per_thread=r, warps_per_cta=8, cull=1, tape_hits=-1) for r in table]
    path = str(tmp_path / "c.json")
    import paper_2509_10247_b300.autotune as at
    orig = at._equal
    at._equal = lambda a, b: a == b
    try:
        e = autotune.tune(p, inp, cands=cands, path=path, runner=runner, gpu_name="fake", ckpts=[])
    finally:
        at._equal = orig
    assert e["exec"]["rays_per_thread"] == 3 and e["ms"] == 2.0 and e["default_ms"] == 9.0
    assert e["tried"] == 5 and e["admitted"] == 3
    assert {x["rays_per_thread"] for x in e["rejected"]} == {2, 4}
    # cached: a second call does not run anything
    e2 = autotune.tune(p, inp, cands=cands, path=path, runner=None, gpu_name="fake", ckpts=[])
    assert e2 == json.loads(json.dumps(e))
    # another GPU name misses the cache
    with pytest.raises(RuntimeError):
        autotune.tune(p, inp, cands=cands, path=path, runner=lambda ex: (None, None), gpu_name="other", ckpts=[])


def test_select_ties_are_deterministic():
    a = {"exec": {"rays_per_thread": 4}, "ms": 1.0, "ok": True}
    b = {"exec": {"rays_per_thread": 2}, "ms": 1.0, "ok": True}
    assert autotune.select([a, b]) is b and autotune.select([b, a]) is b
    assert autotune.select([dict(a, ok=False)]) is None


def test_candidates_are_valid_configs():
    from paper_2509_10247_b300 import binding
    p, _ = _wl()
    modes = set()
    for ex in autotune.candidates(p):
        cfg = binding.make_config(p, **ex)
        assert cfg.rays_per_thread in (0, 1, 2, 3, 4, 5, 6, 8)
        assert cfg.cull in (1, 2) and cfg.warps_per_cta in (4, 8)
        assert cfg.cast_mode in (0, 1)
        modes.add(cfg.cast_mode)
    assert modes == {0, 1}
    ks = autotune.ckpt_candidates(p)
    assert ks[0] == 1 and ks[-1] == p["horizon"] and all(1 <= k <= p["horizon"] for k in ks)


def test_second_stage_tunes_the_checkpoint_interval(tmp_path):
    """Stage 2 varies ckpt_every around the best render shape; a faster
    interval that changes the results is not admitted."""
    p, inp = _wl()
    ref = [7]

    def runner(ex):
        k = ex["ckpt_every"]
        if ex["rays_per_thread"] == 2:
            return {1: 3.0, 2: 2.5, 4: 1.5, 16: 2.0}.get(k, 9.0), ([8] if k == 2 else ref)
        return 5.0, ref

    import paper_2509_10247_b300.autotune as at
    orig = at._equal
    at._equal = lambda a, b: a == b
    try:
        cands = [dict(rays_per_thread=r, warps_per_cta=8, cull=1, tape_hits=-1) for r in (1, 2)]
        e = autotune.tune(p, inp, cands=cands, path=str(tmp_path / "k.json"), runner=runner, gpu_name="fake",
                          ckpts=[1, 2, 4, 16])
    finally:
        at._equal = orig
    assert e["exec"]["rays_per_thread"] == 2 and e["exec"]["ckpt_every"] == 4 and e["ms"] == 1.5
    assert {"rays_per_thread": 2, "warps_per_cta": 8, "cull": 1, "tape_hits": -1, "ckpt_every": 2} in e["rejected"]
