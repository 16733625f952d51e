"""Host side of the launch-shape autotuner: the cache key and the JSON cache
round trip, and the C struct <-> dict conversion (no GPU needed)."""

import json

from paper_2104_06336_gb300 import _lib as L
from paper_2104_06336_gb300 import tuning
import synth


def test_cache_key_separates_geometry_precision_and_device():
    g1 = synth.geometry(synth.workload(1))
    g2 = synth.geometry(synth.workload(1, scan_ny=64, scan_nx=64))
    k = tuning.cache_key(g1, 0, "GPU A")
    assert k == tuning.cache_key(dict(g1), 0, "GPU A")
    assert k != tuning.cache_key(g2, 0, "GPU A")
    assert k != tuning.cache_key(g1, 1, "GPU A")
    assert k != tuning.cache_key(g1, 0, "GPU B")


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert tuning.load_cache(path) == {}
    t = {"scatter_tf": 32, "scatter_ctas_per_sm": 2, "dft_ctas_per_sm": 4,
         "trotter_ctas_per_sm": 3, "ms": [0.4, 1.8, 0.77]}
    tuning.store_cache(path, "k1", t)
    tuning.store_cache(path, "k2", dict(t, scatter_tf=64))
    d = tuning.load_cache(path)
    assert d["k1"] == t and d["k2"]["scatter_tf"] == 64
    (tmp_path / "bad.json").write_text("not json")
    assert tuning.load_cache(str(tmp_path / "bad.json")) == {}
    json.loads(open(path).read())


def test_tuning_struct_conversion():
    t = {"scatter_tf": 16, "scatter_ctas_per_sm": 1, "dft_ctas_per_sm": 2,
         "trotter_ctas_per_sm": 3, "ms": [1.0, 2.0, 3.0]}
    assert L.Tuning.from_dict(t).as_dict() == t
    assert L.Tuning.from_dict({}).as_dict()["scatter_tf"] == 0
