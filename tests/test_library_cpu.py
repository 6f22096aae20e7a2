"""Host-side checks of the CUDA library that need no GPU: it builds for
sm_103a, loads, and exports every entry point include/lf.h declares."""
import json
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^[a-z_0-9 \*]+?\b(lf_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2402_14670_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    d = _declared()
    for n in ("lf_create", "lf_destroy", "lf_pack_hits", "lf_find_tracks", "lf_find_tracks_batched",
              "lf_last_error", "lf_sync_status", "lf_debug_stages", "lf_device_sm_count"):
        assert n in d


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_path]).decode()
    exported = set(re.findall(r"\bT (lf_[a-z_0-9]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match(lib_path):
    from paper_2402_14670_gb300 import lf
    assert sorted(lf.EXPORTED) == sorted(n for n in _declared() if n in lf.EXPORTED)
    for n in _declared():
        assert hasattr(lf, n), n


def test_library_defaults_are_the_papers_constants():
    from paper_2402_14670_gb300 import lf
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    p = lf.default_params()
    for k, v in gold["forward_tolerances"].items():
        if not k.startswith("_"):
            assert p[k] == v, k
    assert p["C_n"] == [gold["C_n"][str(n)] for n in (9, 10, 11, 12)]
    pk = lf.default_params(paper_K=True)
    assert pk["K_first"] == gold["K_x1"]["K_first"] and pk["K_last"] == gold["K_x1"]["K_last"]
    assert lf.default_geometry()["z_ref"] == gold["z_ref_mm"]["value"]


def test_library_and_oracle_defaults_agree():
    import oracle
    from paper_2402_14670_gb300 import lf
    assert lf.default_params() == oracle.default_params()
    assert lf.default_params(True) == oracle.default_params(True)
    assert lf.default_geometry() == oracle.default_geometry()


def test_tensor_layer_refuses_host_tensors():
    import torch
    from paper_2402_14670_gb300 import lf
    with pytest.raises(ValueError):
        lf._ptr(torch.zeros(4))
