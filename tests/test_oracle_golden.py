"""The oracle's parameter defaults equal the values the paper prints (App. B)."""
import json
import os

import pytest

HERE = os.path.dirname(__file__)


def test_defaults_match_paper(oracle_mod):
    with open(os.path.join(HERE, "golden", "app_b_defaults.json")) as f:
        gold = json.load(f)
    p = oracle_mod.default_params()
    for k, v in gold.items():
        if k.startswith("_"):
            continue
        assert p[k] == pytest.approx(v["value"], rel=0, abs=0), (k, v["cite"])
