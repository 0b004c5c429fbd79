"""The autotuner's host logic on the CPU, with the timing faked: the
configurations it tries per storage, the choice of the fastest, and the
per-device cache (stored after a measurement, reused after it, refreshed on
retune).  No GPU is touched."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_1203_6350_gb300 import autotune  # noqa: E402


def test_configurations_per_storage():
    f64 = autotune.configurations("f64")
    assert f64 and all(c[:2] == (1, 1) for c in f64)  # one cell per thread only
    assert len(f64) == len(autotune.CANDIDATES)
    f32 = autotune.configurations("f32")
    two = [c for c in f32 if c[1] == 2]
    assert two == [(2, 2) + autotune.TWO_STEP_TILE]  # the two-step tile is fixed
    assert len(f32) == 2 * len(autotune.CANDIDATES) + 1


def test_fastest_configuration_is_cached_per_device(monkeypatch, tmp_path):
    monkeypatch.setenv("LBM_AUTOTUNE_CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "Fake GPU")
    calls = []

    def fake_measure(shapes, storage, configs=None):
        calls.append(storage)
        cfgs = autotune.configurations(storage)
        # the two-step kernel fastest, then pairs on 128 x 8 tiles
        return {c: (1e-4 if c[1] == 2 else 2e-4 if c[:2] == (2, 1) and c[2:] == (128, 8)
                    else 3e-4) for c in cfgs}

    monkeypatch.setattr(autotune, "measure", fake_measure)
    shapes = [(100, 60), (300, 70)]
    got = autotune.tuned_config(shapes, "f32")
    assert got == {"cells": 2, "steps_per_launch": 2, "tile": autotune.TWO_STEP_TILE}
    assert calls == ["f32"]
    # reused from the cache, for the same shape signature in any order
    assert autotune.tuned_config([(310, 65), (99, 61)], "f32") == got and calls == ["f32"]
    cache = json.loads((tmp_path / "autotune.json").read_text())
    (key,) = cache
    assert key.startswith("Fake GPU|f32|") and len(cache[key]["seconds_per_step"]) == len(
        autotune.configurations("f32"))
    # another storage is another entry; retune measures again
    assert autotune.tuned_config(shapes, "f64")["cells"] == 1
    autotune.tuned_config(shapes, "f32", retune=True)
    assert calls == ["f32", "f64", "f32"]
