"""The tensor-core sign kernel's bounded waits, made to run out on purpose (no fault, no hang).

Every wait of one warp role on another in the kernel is bounded (options.wait_ns, 2 s by default). With a
limit of 1 ns the waits give up at once: the kernel takes its timeout exit (waits for its own copies and
products in flight, frees its tensor memory, returns), the submatrices in flight and those no block took
report NOLSM_ERR_TIMEOUT, the call returns that status, and the device stays usable: the next solve with the
default limit matches the FP64 oracle."""
import numpy as np
import pytest

from oracle import nolsm_oracle as orc
from synth import make_system, spec_small_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    return nl


@pytest.mark.parametrize("prec", ["bf16x3", "fp16"])
def test_a_wait_that_runs_out_is_reported_and_the_device_stays_usable(nl, prec):
    sysm = make_system(spec_small_fp64())
    ref = orc.solve(sysm, -0.1)
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    nl.nolsm_solve_batch(plan, -0.1, nl.options(prec))   # geometry prepared with the default limit
    r = nl.nolsm_solve_batch(plan, -0.1, nl.options(prec, wait_ns=1), check=False)
    st = r.sub_status.cpu().numpy()
    timed_out = int(np.sum(st == nl._abi.ERR_TIMEOUT))
    print(f"{prec}, 1 ns wait limit: status {r.status}, {timed_out} of {sysm.n_mol} submatrices timed out")
    assert r.status == nl._abi.ERR_TIMEOUT
    assert timed_out > 0
    assert set(np.unique(st).tolist()) <= {0, nl._abi.ERR_TIMEOUT}
    # the next solve with the default limit is complete and correct
    r2 = nl.nolsm_solve_batch(plan, -0.1, nl.options(prec))
    D = plan.scatter().cpu().numpy()
    err = float(np.max(np.abs(D - ref.D_vals)))
    assert r2.status == 0 and np.all(r2.sub_status.cpu().numpy() == 0)
    assert err <= 1e-4
    plan.close()
