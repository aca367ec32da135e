"""Host-side logic of the batched form's autotuner: the workload key and the
cached choice, which is returned without timing anything."""

import json
from types import SimpleNamespace

import torch

from paper_2504_06598_gb300 import autotune


def _workload(M=1000, deg=3, dtype=torch.float32, sizes=((64, 32), (16, 16)), lights=2, bounce=1):
    g = SimpleNamespace(M=M, sh_degree=deg, sh=torch.zeros(1, dtype=dtype))
    cams = [SimpleNamespace(width=w, height=h) for w, h in sizes]
    ex = SimpleNamespace(lights=[None] * lights, bounce=bounce)
    return g, cams, ex


def test_key_names_every_shape_that_changes_the_choice():
    g, cams, ex = _workload()
    k = autotune.workload_key(g, cams, ex, spp=4)
    assert k == "M1000_deg3_shfloat32_v2_px2304_spp4_l2_b1"
    variants = [
        autotune.workload_key(*_workload(M=1001)[:2], ex, spp=4),
        autotune.workload_key(*_workload(dtype=torch.float16)[:2], ex, spp=4),
        autotune.workload_key(*_workload(sizes=((64, 32),))[:2], ex, spp=4),
        autotune.workload_key(g, cams, ex, spp=8),
        autotune.workload_key(g, cams, _workload(lights=4)[2], spp=4),
        autotune.workload_key(g, cams, _workload(bounce=0)[2], spp=4),
        autotune.workload_key(g, cams, None, spp=4),
    ]
    assert len(set(variants + [k])) == len(variants) + 1


def test_cached_choice_is_returned_without_timing(tmp_path, monkeypatch):
    g, cams, ex = _workload()
    key = autotune.workload_key(g, cams, ex, spp=4)
    choice = {"node_format": "wide4_q8", "stack_entries": 96, "block_threads": 128, "ms": 1.5,
              "key": key}
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({key: choice}))

    def no_gpu(*a, **k):
        raise AssertionError("a cached workload must not be timed")

    monkeypatch.setattr(autotune, "build_bvh", no_gpu)
    monkeypatch.setattr(autotune, "render_views", no_gpu)
    res = autotune.autotune(g, cams, ex, spp=4, cache_path=str(path))
    assert res["cached"] is True
    assert {k: res[k] for k in choice} == choice
