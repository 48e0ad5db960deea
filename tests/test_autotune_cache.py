"""The autotuner's cache (host logic, no GPU): shape classes, and the winner
stored and found again per GPU name and class in the JSON file that
MT_AUTOTUNE_CACHE names."""

from __future__ import annotations

import json

import pytest

from paper_2301_10838_gb300 import autotune


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("MT_AUTOTUNE_CACHE", str(path))
    names = {0: "GPU-A", 1: "GPU-B"}
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda d: names[int(d)])
    return path


def test_shape_classes():
    assert autotune.single_class((1024, 1024, 1024)) == "single-n30-x10-f0"
    assert autotune.single_class((1024, 1024, 1024), flags=1) == "single-n30-x10-f1"
    # grids of about the same size and x side share a class; others do not
    assert autotune.single_class((1000, 1030, 1024)) == autotune.single_class((1024, 1024, 1024))
    assert autotune.single_class((64, 64, 64)) != autotune.single_class((256, 256, 256))
    assert autotune.single_class((4096, 512, 512)) != autotune.single_class((512, 512, 4096))
    shapes = [(16, 16, 16)] * 3 + [(32, 32, 32)]
    assert autotune.batch_class(shapes) == "batch-n4-mean13-max15"


def test_store_and_lookup_per_gpu_and_class(cache):
    assert autotune.lookup(0, "single-n30-x10-f0") is None  # no file yet
    autotune.store(0, "single-n30-x10-f0", 8, {"0": 49.5, "8": 51.6})
    autotune.store(0, "batch-n512-mean17-max20", 1, [5.6, 6.9])
    hit = autotune.lookup(0, "single-n30-x10-f0")
    assert hit == {"cfg": 8, "ms": {"0": 49.5, "8": 51.6}}
    assert autotune.lookup(0, "batch-n512-mean17-max20")["cfg"] == 1
    assert autotune.lookup(1, "single-n30-x10-f0") is None  # another GPU
    assert autotune.lookup(0, "single-n20-x7-f0") is None   # another class
    autotune.store(0, "single-n30-x10-f0", 0, {"0": 49.0})  # a later tuning replaces it
    assert autotune.lookup(0, "single-n30-x10-f0")["cfg"] == 0
    on_disk = json.loads(cache.read_text())
    assert set(on_disk) == {"GPU-A|single-n30-x10-f0", "GPU-A|batch-n512-mean17-max20"}


def test_unreadable_cache_is_a_miss(cache):
    cache.write_text("{not json")
    assert autotune.lookup(0, "single-n30-x10-f0") is None
    autotune.store(0, "single-n30-x10-f0", 2, {"2": 1.0})  # rewrites the file
    assert autotune.lookup(0, "single-n30-x10-f0")["cfg"] == 2
