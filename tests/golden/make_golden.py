"""Writes the oracle's regression fixtures in this folder. Calls only ``oracle/`` (and the seeded
inputs of ``synth/``); run it after a change to the oracle's arithmetic that a passage of the paper
justifies, and name that passage in the commit.

    python tests/golden/make_golden.py

The paper prints no worked numeric example (its numbers are throughputs on systems whose inputs are not
available), so nothing here is the paper's own value: these fixtures only freeze what the pinned oracle
computes, so that an unintended change to it shows up as a failing test."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import combine_oracle as co  # noqa: E402
from oracle import nolsm_oracle as orc  # noqa: E402
from synth import make_site_pattern, make_system, spec_ions_in_water_small, spec_small_fp64  # noqa: E402


def small_fp64():
    sysm = make_system(spec_small_fp64())
    res = orc.solve(sysm, -0.1)
    w = orc.energy_weighted(sysm, res)
    J = 17
    return {"system": "64 molecules (4x4x4), 6 functions each, seed 1001, mu = -0.1",
            "trace_DS": res.trace_DS, "trace_DH": res.trace_DH, "trace_WS": w.trace_WS,
            "steps": " ".join(str(int(res.subs[j].steps)) for j in range(sysm.n_mol)),
            "D_cols_17_first_row": [float(x) for x in res.subs[J].D_cols[0]],
            "D_vals_sum": float(res.D_vals.sum()), "D_vals_abs_sum": float(abs(res.D_vals).sum())}


def ions_small():
    sp = make_site_pattern(spec_ions_in_water_small())
    r = co.combine(sp.nbf, sp.nb_ptr, sp.nb_idx)
    return {"pattern": "atom-resolved water 6x6x6 with 3 % ions, seed 1302",
            "sites": sp.n_sites, "groups": len(r.members), "sweeps": r.sweeps, "merges": len(r.merges),
            "sum_n3_before": r.sum_n3_before, "sum_n3_after": r.sum_n3_after,
            "sum_n2_before": r.sum_n2_before, "sum_n2_after": r.sum_n2_after}


if __name__ == "__main__":
    out = {"oracle_small_fp64": small_fp64(), "combine_ions_small": ions_small()}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
