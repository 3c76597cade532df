"""The stored oracle values are well-formed: the fixtures that the full-size
GPU parity tests read (tests/golden/kb1024_oracle.json and
kb1024_clean_oracle.json, written by make_kb1024_oracle.py, and
mixed2048_oracle.json, written by make_mixed2048_oracle.py, from oracle/ and
synth/ only) and the paper's printed parameters."""
import json
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name", ["kb1024_oracle.json", "kb1024_clean_oracle.json"])
def test_kb1024_oracle_fixture_is_complete(name):
    g = json.load(open(os.path.join(HERE, name)))
    assert g["sample_columns"] == ["y", "x", "disp", "probe"]
    assert g["probes"] == ["images", "state", "all", "noise1", "noise2"]
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
    assert 0 < ps["mean"] <= ps["q998"] <= ps["max"] <= g["probe_field_stats"]["max"]
    assert g["n_mask"] == 1024 * 1024 and g["gt_errors"]["n"] == g["n_mask"]
    # both fixtures sample the same pixels of the same scene
    other = json.load(open(os.path.join(HERE, "kb1024_oracle.json")))
    assert [r[:2] for r in other["sample"]] == [r[:2] for r in g["sample"]]


def test_mixed2048_oracle_fixture_is_complete():
    g = json.load(open(os.path.join(HERE, "mixed2048_oracle.json")))
    assert g["sample_columns"] == ["y", "x", "disp", "probe_fp32", "probe_fp16", "probe_bf16"]
    assert (g["levels"], g["warps"], g["iters"]) == (6, 2, 20)
    s = np.array(g["sample"], dtype=np.float64)
    assert s.shape == (8192, 6) and np.isfinite(s).all() and (s[:, 3:] >= 0).all()
    y, x = s[:, 0].astype(int), s[:, 1].astype(int)
    assert y.min() >= 0 and x.min() >= 0 and y.max() < 2048 and x.max() < 2048
    assert len(set(zip(y.tolist(), x.tolist()))) == 8192
    # reach of the clipped increments: 0.2 px x 2 warps x (2^6 - 1)
    assert np.abs(s[:, 2]).max() <= 0.2 * 2 * 63
    pf = g["probe_field"]
    # coarser storage, larger response: fp32 < fp16 < bf16
    assert pf["fp32"]["mean"] < pf["fp16"]["mean"] < pf["bf16"]["mean"]


def test_paper_parameters_fixture_cites_the_paper():
    g = json.load(open(os.path.join(HERE, "paper_parameters.json")))
    for k, v in g.items():
        if isinstance(v, dict):
            assert "value" in v and v.get("cite", "").startswith("Sec."), k
    # the TGV weights of Sec. IV-C are the oracle's defaults too
    import oracle
    prm = oracle.Params()
    assert prm.alpha0 == g["alpha0"]["value"] and prm.alpha1 == g["alpha1"]["value"]


def test_every_oracle_function_cites_its_passage():
    # each function of the oracle names the section, equation or algorithm of
    # the paper it follows
    import ast
    import glob
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    missing = []
    for f in sorted(glob.glob(os.path.join(root, "oracle", "*.py"))):
        for n in ast.parse(open(f).read()).body:
            if isinstance(n, ast.FunctionDef):
                d = ast.get_docstring(n) or ""
                if not any(k in d for k in ("Sec.", "Eq.", "Algorithm")):
                    missing.append(f"{os.path.basename(f)}:{n.name}")
    assert not missing, missing


def test_profile_summaries_are_text_and_name_committed_commands():
    # profiles/ holds short text summaries only, and every command they give
    # runs a module or script of this repository
    import re
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pdir = os.path.join(root, "profiles")
    names = sorted(os.listdir(pdir))
    assert names and all(n.endswith((".md", ".txt")) for n in names), names
    try:
        tracked = set(subprocess.run(["git", "ls-files"], cwd=root, capture_output=True,
                                     text=True).stdout.split())
    except OSError:                   # no git: check the files exist instead
        tracked = set()
    for n in names:
        text = open(os.path.join(pdir, n)).read()
        assert len(text) < 16384, n
        cmds = re.findall(r"python -m ([\w.]+)|python ([\w/]+\.py)", text)
        assert cmds, f"{n} gives no command"
        for mod, script in cmds:
            path = mod.replace(".", "/") + ".py" if mod else script
            if tracked:
                assert path in tracked, (n, path)
            else:
                assert os.path.exists(os.path.join(root, path)), (n, path)


def test_fixture_scripts_use_only_the_oracle_and_the_input_generators():
    # the stored expected values are written by scripts that import the
    # oracle and the seeded inputs, never the CUDA path or torch
    import ast
    import glob
    allowed = {"oracle", "synth", "numpy", "json", "multiprocessing", "os", "sys", "time",
               "math", "argparse", "__future__", "hashlib"}
    scripts = sorted(glob.glob(os.path.join(HERE, "make_*.py")))
    assert scripts
    for f in scripts:
        tree = ast.parse(open(f).read())
        for n in ast.walk(tree):
            if isinstance(n, ast.Import):
                mods = [a.name.split(".")[0] for a in n.names]
            elif isinstance(n, ast.ImportFrom):
                mods = [(n.module or "").split(".")[0]]
            else:
                continue
            for m in mods:
                assert m in allowed, (os.path.basename(f), m)


def test_oracle_and_gpu_path_import_nothing_of_each_other():
    # the oracle imports neither the library nor torch; the library's package
    # imports no oracle; the seeded inputs import neither
    import ast
    import glob
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    banned = {"oracle": {"paper_1909_07545_gb300", "torch"},
              "paper_1909_07545_gb300": {"oracle"},
              "synth": {"oracle", "paper_1909_07545_gb300", "torch"}}
    for pkg, bad in banned.items():
        for f in sorted(glob.glob(os.path.join(root, pkg, "*.py"))):
            for n in ast.walk(ast.parse(open(f).read())):
                if isinstance(n, ast.Import):
                    mods = [a.name.split(".")[0] for a in n.names]
                elif isinstance(n, ast.ImportFrom) and n.level == 0:
                    mods = [(n.module or "").split(".")[0]]
                else:
                    continue
                for m in mods:
                    assert m not in bad, (pkg, os.path.basename(f), m)
