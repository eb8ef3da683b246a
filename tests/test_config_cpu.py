"""A session's configuration survives JSON exactly (base graphs, lifting sizes, arithmetic), and a tampered
base graph is refused."""
import json

import numpy as np
import pytest

from paper_2506_00167_gb300 import config
from workload.configs import default_bgs


def test_configuration_round_trips_through_json():
    bgs = default_bgs()
    cfg = config.session_config(bgs, [32, 64, 384], mode="i8", max_iter=8, early_term=False, q_scale=4.0)
    text = config.dumps(cfg)
    graphs, z_set, kw = config.loads(text)
    assert z_set == [32, 64, 384]
    assert kw == {"mode": "i8", "max_iter": 8, "early_term": False, "offset_f32": 0.5, "offset_lsb": 1,
                  "q_scale": 4.0, "interleave": True, "sat": (63, 63, 127)}  # defaults made explicit
    for g, h in zip(bgs, graphs):
        assert (g.mb, g.nb, g.kb, g.mc, g.n_punct_cols) == (h.mb, h.nb, h.kb, h.mc, h.n_punct_cols)
        for a in ("row", "col", "V"):
            assert np.array_equal(np.asarray(getattr(g, a), np.int16), getattr(h, a))
    # writing the loaded configuration again gives the same text
    again = config.session_config(graphs, z_set, **kw)
    assert config.dumps(again) == text


def test_tampered_graph_and_unknown_version_are_refused():
    cfg = json.loads(config.dumps(config.session_config(default_bgs(), [64])))
    cfg["base_graphs"][0]["entries"][5][2] += 1
    with pytest.raises(ValueError, match="SHA-256"):
        config.session_args(cfg)
    cfg = config.session_config(default_bgs(), [64])
    cfg["version"] = 99
    with pytest.raises(ValueError, match="version"):
        config.session_args(cfg)
    with pytest.raises(ValueError, match="mode"):
        config.session_config(default_bgs(), [64], mode="f16")
