"""The oracle against its frozen outputs (tests/golden/oracle_regression.json, written by
tests/golden/make_golden.py from the oracle alone). Not a pin: the pins are the closed forms and
invariants of the *_pins tests; this catches an unintended change to the oracle's arithmetic."""
import json
import os

import pytest

from oracle import combine_oracle as co
from oracle import nolsm_oracle as orc
from synth import make_site_pattern, make_system, spec_ions_in_water_small, spec_small_fp64

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_regression.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_small_system_solve(golden):
    g = golden["oracle_small_fp64"]
    sysm = make_system(spec_small_fp64())
    res = orc.solve(sysm, -0.1)
    w = orc.energy_weighted(sysm, res)
    assert res.trace_DS == pytest.approx(g["trace_DS"], abs=1e-12)
    assert res.trace_DH == pytest.approx(g["trace_DH"], abs=1e-12)
    assert w.trace_WS == pytest.approx(g["trace_WS"], abs=1e-12)
    assert " ".join(str(int(res.subs[j].steps)) for j in range(sysm.n_mol)) == g["steps"]
    assert list(res.subs[17].D_cols[0]) == pytest.approx(g["D_cols_17_first_row"], abs=1e-14)
    assert float(res.D_vals.sum()) == pytest.approx(g["D_vals_sum"], abs=1e-11)
    assert float(abs(res.D_vals).sum()) == pytest.approx(g["D_vals_abs_sum"], abs=1e-11)


def test_combination_on_ions_in_water(golden):
    g = golden["combine_ions_small"]
    sp = make_site_pattern(spec_ions_in_water_small())
    r = co.combine(sp.nbf, sp.nb_ptr, sp.nb_idx)
    got = {"sites": sp.n_sites, "groups": len(r.members), "sweeps": r.sweeps, "merges": len(r.merges),
           "sum_n3_before": r.sum_n3_before, "sum_n3_after": r.sum_n3_after,
           "sum_n2_before": r.sum_n2_before, "sum_n2_after": r.sum_n2_after}
    assert got == {k: g[k] for k in got}
