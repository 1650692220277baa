"""Selection and caching logic of the autotuner, with a fake timing function (no GPU)."""
import json
import math

from paper_0805_3041_gb300 import autotune, inputs


def spec(n, eps):
    return inputs.anisotropic(n=n, eps=eps)


def test_class_key_buckets_anisotropy_by_half_decade():
    assert autotune.class_key(spec(65, 1.0)) == "65x65:eps1e+0.0"
    assert autotune.class_key(spec(65, 0.3)) == "65x65:eps1e-0.5"
    assert autotune.class_key(spec(129, 1e-3)) == "129x129:eps1e-3.0"
    assert autotune.class_key(spec(129, 1.2e-3)) == autotune.class_key(spec(129, 1e-3))


def test_tune_picks_fastest_converging_schedule_then_knobs():
    calls = []

    def measure(sp, cfg):
        calls.append(dict(cfg))
        if cfg["smoother"] == "rbgs":
            return math.inf                       # does not converge (strong anisotropy)
        t = {"zebra_y": 2.0, "line_y": 3.0, "gsadi": 2.5, "adi": 4.0}[cfg["smoother"]] + 0.1 * cfg["nu1"]
        if cfg.get("tile_nodes") == -1:
            t -= 0.05
        return t

    tu = autotune.Autotuner(measure=measure)
    cfg, trials = tu.tune(spec(129, 1e-3))
    assert cfg["smoother"] == "zebra_y" and cfg["nu1"] == 1 and cfg["tile_nodes"] == -1
    assert len(trials) == len(autotune.SCHEDULES) + len(autotune.KNOBS) - 1
    # cached: choose() does not time again
    n = len(calls)
    assert tu.choose(spec(129, 1.1e-3)) == cfg
    assert len(calls) == n


def test_nothing_converges_keeps_default():
    tu = autotune.Autotuner(measure=lambda sp, cfg: math.inf)
    cfg, _ = tu.tune(spec(65, 1.0))
    assert cfg == autotune.DEFAULT
    assert tu.table[autotune.class_key(spec(65, 1.0))]["seconds"] is None


def test_table_round_trip(tmp_path):
    tu = autotune.Autotuner(measure=lambda sp, cfg: 1.0 + 0.1 * cfg["nu1"] + (0.5 if cfg["smoother"] != "rbgs" else 0))
    tu.tune(spec(65, 1.0))
    p = tmp_path / "t.json"
    tu.save(str(p))
    data = json.loads(p.read_text())
    assert "65x65:eps1e+0.0" in data["classes"]
    tu2 = autotune.Autotuner(path=str(p), measure=lambda sp, cfg: 1 / 0)   # must not be called
    assert tu2.choose(spec(65, 1.0)) == tu.choose(spec(65, 1.0))
