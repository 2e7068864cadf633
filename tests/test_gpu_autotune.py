"""The launch-shape tuner of the tensor-core kernel (no counterpart in the paper, which calls library GEMMs).

The kernel has two launch shapes (0: 384 threads, tiles of 128 x up to 256 columns; 1: 512 threads with three
epilogue groups and a register split, tiles of 128 x up to 192). Every solve of the sign iteration and every
preparation chunk of the inverse square root splits its submatrices into n > 192 and n <= 192 buckets; the
shape of a (kernel, precision, bucket) is measured the first time a process meets it, or fixed by the
environment variable NOLSM_TC_SHAPE. Checked here on the 4,096-molecule uneven system (n 138-240, so both
buckets are used): either fixed shape gives every submatrix a converged status and the same density within
twice the BF16X3 mode's measured error (both are about 6e-7 from the FP64 oracle, which the parity tests
check), and with the tuner on, its choice for every bucket it met is one of the two shapes and the density
agrees as well."""
import os

import numpy as np
import pytest

from synth import make_system, spec_batched_uneven_4096

pytestmark = pytest.mark.gpu

TOL_SHAPES = 5e-6


@pytest.fixture(scope="module")
def nl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    return nl


@pytest.fixture(scope="module")
def system():
    return make_system(spec_batched_uneven_4096())


def _solve(nl, system, shape):
    """One solve at mu = -0.35 on a fresh plan (its preparation included) with NOLSM_TC_SHAPE set to shape
    (None: unset, the tuner decides)."""
    old = os.environ.get("NOLSM_TC_SHAPE")
    if shape is None:
        os.environ.pop("NOLSM_TC_SHAPE", None)
    else:
        os.environ["NOLSM_TC_SHAPE"] = str(shape)
    try:
        plan = nl.nolsm_build_submatrices(nl.DeviceSystem(system))
        o = nl.options("bf16x3", inverse=nl._abi.INVERSE_NEWTON_SCHULZ)
        r = nl.nolsm_solve_batch(plan, -0.35, o)
        D = plan.scatter().cpu().numpy()
        plan.close()
        return r, D
    finally:
        if old is None:
            os.environ.pop("NOLSM_TC_SHAPE", None)
        else:
            os.environ["NOLSM_TC_SHAPE"] = old


def test_both_shapes_give_the_same_density(nl, system):
    assert np.any(system.nbf > 0)
    r0, D0 = _solve(nl, system, 0)
    r1, D1 = _solve(nl, system, 1)
    assert np.all(r0.sub_status.cpu().numpy() == 0)
    assert np.all(r1.sub_status.cpu().numpy() == 0)
    diff = float(np.max(np.abs(D0 - D1)))
    print(f"shape 0 vs shape 1: max|dD| {diff:.2e}, Tr(DS) {r0.trace_DS:.6f} vs {r1.trace_DS:.6f}")
    assert diff <= TOL_SHAPES
    assert abs(r0.trace_DS - r1.trace_DS) <= 1e-6 * abs(r0.trace_DS)


def test_tuner_picks_one_of_the_shapes(nl, system):
    r0, D0 = _solve(nl, system, 0)
    ra, Da = _solve(nl, system, None)
    assert np.all(ra.sub_status.cpu().numpy() == 0)
    choices = {(k, b): nl.nolsm_tc_shape(k, "bf16x3" if k == "sign" else "fp16", b)
               for k in ("sign", "inverse") for b in (0, 1)}
    print("tuned shapes:", choices)
    assert all(v in (0, 1) for v in choices.values())
    assert float(np.max(np.abs(Da - D0))) <= TOL_SHAPES
