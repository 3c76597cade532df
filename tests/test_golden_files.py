"""The stored oracle values are well-formed: the fixture that the full-size
GPU parity test reads (tests/golden/kb1024_oracle.json, written by
make_kb1024_oracle.py from oracle/ and synth/ only) and the paper's printed
parameters."""
import json
import os

import numpy as np

HERE = os.path.join(os.path.dirname(__file__), "golden")


def test_kb1024_oracle_fixture_is_complete():
    g = json.load(open(os.path.join(HERE, "kb1024_oracle.json")))
    assert g["sample_columns"] == ["y", "x", "disp", "probe"]
    s = np.array(g["sample"], dtype=np.float64)
    assert s.shape == (4096, 4)
    y, x = s[:, 0].astype(int), s[:, 1].astype(int)
    assert y.min() >= 0 and x.min() >= 0 and y.max() < 1024 and x.max() < 1024
    assert len(set(zip(y.tolist(), x.tolist()))) == 4096          # distinct pixels
    assert np.isfinite(s).all() and (s[:, 3] >= 0).all()
    q = np.array(g["disp_quantiles"])
    assert len(q) == len(g["quantile_levels"]) == len(g["probe_quantile_shift"])
    assert np.all(np.diff(q) >= 0)
    # the sampled disparities lie within the field's quantile range, and the
    # clipped increments bound the reach: 0.2 px x 10 warps x (2^5 - 1)
    assert s[:, 2].min() >= q[0] - 1.0 and s[:, 2].max() <= 0.2 * 10 * 31
    ps = g["probe_sample_stats"]
    assert 0 < ps["mean"] <= ps["q998"] <= ps["max"]
    assert g["n_mask"] == 1024 * 1024 and g["gt_errors"]["n"] == g["n_mask"]


def test_paper_parameters_fixture_cites_the_paper():
    g = json.load(open(os.path.join(HERE, "paper_parameters.json")))
    for k, v in g.items():
        if isinstance(v, dict):
            assert "value" in v and v.get("cite", "").startswith("Sec."), k
    # the TGV weights of Sec. IV-C are the oracle's defaults too
    import oracle
    prm = oracle.Params()
    assert prm.alpha0 == g["alpha0"]["value"] and prm.alpha1 == g["alpha1"]["value"]
