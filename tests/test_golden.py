"""Fixtures under tests/golden/ (text, each line cited): the values the paper
fixes against the defaults of the library and the oracle, and hand-worked
cases of Algorithm 1 against the host-side selection.  CPU only."""
import os

import oracle
from paper_2512_20943_b300 import RasterConfig
from paper_2512_20943_b300 import pruning
from paper_2512_20943_b300.pruning import select_pruning_level

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _parameters():
    out = {}
    with open(os.path.join(GOLDEN, "paper_parameters.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (x.strip() for x in line.split("="))
                out[k] = float(v)
    return out


def test_defaults_use_the_papers_values():
    p = _parameters()
    cfg = RasterConfig()
    assert cfg.alpha_max == p["alpha_max"] and abs(cfg.alpha_min - p["alpha_min"]) < 1e-15
    assert cfg.T_min == p["T_min"]
    s = oracle.DEFAULT_SETTINGS
    assert s["alpha_max"] == p["alpha_max"] and abs(s["alpha_min"] - p["alpha_min"]) < 1e-15
    assert s["T_min"] == p["T_min"]
    assert pruning.BETA == p["beta_cliff"]
    fr = pruning.pruning_level_space.__defaults__[0]
    assert len(fr) == p["pruning_level_count"]
    assert all(abs(fr[i] - i * p["pruning_level_step"]) < 1e-12 for i in range(len(fr)))
    assert pruning.UPDATE_CHANNELS == p["update_channels"]
    import inspect
    from paper_2512_20943_b300 import Rasterizer
    assert inspect.signature(Rasterizer.l3dgs_loss).parameters["lam"].default == p["lambda_dssim"]


def test_algorithm1_hand_worked_cases():
    n = 0
    with open(os.path.join(GOLDEN, "algorithm1_cases.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            q, s, beta, B, R, level, _ = (x.strip() for x in line.split("|"))
            space = list(zip((float(x) for x in q.split(",")), (float(x) for x in s.split(","))))
            got = select_pruning_level(space, float(beta), float(B), float(R))
            assert got == int(level), (line, got)
            n += 1
    assert n == 8
