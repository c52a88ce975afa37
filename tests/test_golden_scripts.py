"""The stored oracle results and the scripts that wrote them stay in step: the
Laplace-sweep file carries its script's configuration, its sigma is the
least-squares slope of its own drops (Eq. 22), and the script still runs
(on a cut-down case: the stored run is 2x10^10 lattice updates)."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _laplace_doc():
    with open(os.path.join(HERE, "golden", "laplace_oracle_256.json")) as fh:
        return json.load(fh)


def test_laplace_golden_carries_its_script_configuration():
    from tests.golden import make_laplace_oracle as M
    doc = _laplace_doc()
    assert doc["L"] == M.L and doc["steps"] == M.STEPS and doc["window"] == [M.SPAN, M.EVERY]
    assert doc["t_over_tc"] == M.TR and doc["A"] == M.A and doc["s"] == M.S
    assert sorted(doc["fits"]) == sorted(str(k) for k in M.KAPPAS)
    for fit in doc["fits"].values():
        assert sorted(fit["drops"], key=int) == [str(r) for r in M.RADII]


def test_laplace_golden_sigma_is_the_slope_of_its_drops():
    """Eq. 22: Delta p = sigma / R; the stored sigma and intercept are the
    least-squares line through the stored (1/R_eq, Delta p) points, and the
    stored phase densities their means."""
    doc = _laplace_doc()
    for fit in doc["fits"].values():
        drops = list(fit["drops"].values())
        inv_r = np.array([1.0 / d["R_eq"] for d in drops])
        dp = np.array([d["dp"] for d in drops])
        slope, icpt = np.polyfit(inv_r, dp, 1)
        assert abs(slope / fit["sigma"] - 1) < 1e-9 and abs(icpt - fit["intercept"]) < 1e-12
        assert abs(np.mean([d["rho_in"] for d in drops]) - fit["rho_l"]) < 1e-15
        assert abs(np.mean([d["rho_out"] for d in drops]) - fit["rho_g"]) < 1e-15
        assert fit["r2"] > 0.999
    # kappa = 0.5 halves sigma (Eq. 28) within the tolerance of the paper's Fig. 3 check
    ratio = doc["fits"]["0.5"]["sigma"] / doc["fits"]["0.0"]["sigma"]
    assert abs(ratio - 0.5) < 0.04


def test_laplace_golden_script_runs_on_a_small_case(monkeypatch):
    from tests.golden import make_laplace_oracle as M
    for name, value in (("L", 48), ("STEPS", 60), ("SPAN", 20), ("EVERY", 10)):
        monkeypatch.setattr(M, name, value)
    d = M.drop(0.5, 10, 1)
    assert set(d) == {"dp", "R_eq", "rho_in", "rho_out", "R_drift"}
    assert all(np.isfinite(v) for v in d.values())
    assert d["dp"] > 0 and 7 < d["R_eq"] < 13 and d["rho_in"] > 10 * d["rho_out"]
