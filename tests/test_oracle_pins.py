"""The oracle against what the paper and the mathematics fix (CPU only)."""
import json
import os

import pytest

import oracle
import pins

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.default())


def test_defaults_are_the_papers_constants():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        gold = json.load(f)
    p = oracle.default_params()
    for k, v in gold["forward_tolerances"].items():
        if not k.startswith("_"):
            assert p[k] == v, k
    assert p["C_n"] == [gold["C_n"][str(n)] for n in (9, 10, 11, 12)]
    for k in ("xtol_c", "xtol_p", "x_asym", "uv_tol"):
        assert p[k] == gold["window"][k]
    assert p["magtol_min"] == gold["magnet_tolerance_range_mm"]["min"]
    assert p["magtol_max"] == gold["magnet_tolerance_range_mm"]["max"]
    assert p["p_bend"] == gold["p_bend_GeV"]["value"]
    assert p["min_hits"] == gold["min_hits"]["value"]
    pk = oracle.default_params(paper_K=True)
    assert pk["K_first"] == gold["K_x1"]["K_first"] and pk["K_last"] == gold["K_x1"]["K_last"]
    assert oracle.default_geometry()["z_ref"] == gold["z_ref_mm"]["value"]


def test_no_ut_defaults_are_the_papers_constants():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        gold = json.load(f)
    p = oracle.no_ut_params()
    assert p["no_ut"] == 1
    for k, v in gold["forward_no_ut_tolerances"].items():
        if not k.startswith("_"):
            assert p[k] == v, k
    assert p["tol_c"] == gold["no_ut_poly_tol"]["c"]
    w = gold["no_ut_window"]
    for k in ("p_min", "pt_min", "x_overlap", "uv_tol"):
        assert p[k] == w[k], k
    assert p["magtol_min"] == p["magtol_max"] == w["magtol"]
    # T_uv = max(T_x, 15 (|t_x| + |t_y|)): the floor is the no-UT T_x
    assert p["T_uv_min"] == p["T_x"]
