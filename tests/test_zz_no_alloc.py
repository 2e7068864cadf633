"""The allocation-free entry point (nolsm_sign_noalloc) against the plan-based one.

nolsm_sign_noalloc serves callers that cannot allocate device memory when they need a result; it
runs the tensor-core sign iteration on caller-held inputs with the library's static scratch array.
Here it gets the 64 submatrices of the small water-like system (A_i, centre columns, spectral bounds
prepared on the CPU) and must reproduce, within the BF16X3 tolerance of the other tests, the centre
columns of D and the partial traces that nolsm_solve_batch + nolsm_scatter_density give, and those of
the FP64 oracle, on two calls in a row at different chemical potentials (the second call reuses the
shared scratch)."""
import ctypes

import numpy as np
import pytest

from oracle import nolsm_oracle as orc
from synth import make_system, spec_small_fp64

pytestmark = pytest.mark.gpu

TOL_D = 1e-4        # BF16X3 target, as in test_gpu_tc.py
TOL_TR = 1e-5


def test_noalloc_matches_solve_batch_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    lib = nl._abi.load()

    sysm = make_system(spec_small_fp64())
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    n_mol = sysm.n_mol
    # caller-held inputs, prepared on the CPU in FP64
    A_parts, Q_parts, Sc_parts, Hc_parts, lam = [], [], [], [], []
    a_off, c_off = [0], [0]
    for J in range(n_mol):
        S = orc.gather(po, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
        H = orc.gather(po, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
        c0, b = int(po.sub_c0[J]), int(po.nbf[J])
        A = np.linalg.solve(S, H)
        d = np.diag(A)
        R = np.sum(np.abs(A), axis=1) - np.abs(d)
        lam += [float(np.min(d - R)), float(np.max(d + R))]
        A_parts.append(A.astype(np.float32).ravel())
        Q_parts.append(np.linalg.inv(S)[:, c0:c0 + b].ravel())
        Sc_parts.append(S[:, c0:c0 + b].ravel())
        Hc_parts.append(H[:, c0:c0 + b].ravel())
        a_off.append(a_off[-1] + A.size)
        c_off.append(c_off[-1] + S.shape[0] * b)
    dev = torch.device("cuda")
    T = lambda x, dt: torch.as_tensor(np.asarray(x), dtype=dt).to(dev)
    sub_n, nbf = T(po.sub_n, torch.int32), T(po.nbf, torch.int32)
    aoff, coff = T(a_off[:-1], torch.int64), T(c_off[:-1], torch.int64)
    A_d = T(np.concatenate(A_parts), torch.float32)
    Q_d = T(np.concatenate(Q_parts), torch.float64)
    Sc_d = T(np.concatenate(Sc_parts), torch.float64)
    Hc_d = T(np.concatenate(Hc_parts), torch.float64)
    lam_d = T(lam, torch.float64)

    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    opts = nl.options("bf16x3")
    off = orc.d_block_offsets(po)
    for mu in (-0.1, 0.05):
        ref = nl.nolsm_solve_batch(plan, mu, opts)
        D = plan.scatter().cpu().numpy()
        Dc = torch.full((c_off[-1],), float("nan"), dtype=torch.float64, device=dev)
        tS = torch.zeros(n_mol, dtype=torch.float64, device=dev)
        tH = torch.zeros_like(tS)
        it = torch.zeros(n_mol, dtype=torch.int32, device=dev)
        st = torch.full((n_mol,), -1, dtype=torch.int32, device=dev)
        rc = lib.nolsm_sign_noalloc(n_mol, sub_n.data_ptr(), nbf.data_ptr(), aoff.data_ptr(), coff.data_ptr(),
                                    A_d.data_ptr(), Q_d.data_ptr(), Sc_d.data_ptr(), Hc_d.data_ptr(),
                                    lam_d.data_ptr(), mu, ctypes.byref(opts),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                    Dc.data_ptr(), tS.data_ptr(), tH.data_ptr(), it.data_ptr(), st.data_ptr())
        assert rc == 0, lib.nolsm_last_error().decode()
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy() == 0)
        Dc_h = Dc.cpu().numpy()
        err = 0.0
        for J in range(n_mol):
            b = int(po.nbf[J])
            cols = Dc_h[c_off[J]:c_off[J + 1]].reshape(-1, b)
            for p in range(po.nb_ptr[J], po.nb_ptr[J + 1]):
                I = int(po.nb_idx[p])
                q = po.nb_ptr[I] + int(np.nonzero(po.nb_idx[po.nb_ptr[I]:po.nb_ptr[I + 1]] == J)[0][0])
                blk = D[off[q]:off[q + 1]].reshape(int(po.nbf[I]), b)
                err = max(err, float(np.max(np.abs(blk - cols[po.nb_off[p]:po.nb_off[p] + blk.shape[0], :]))))
        # the FP64 oracle's centre columns and partial traces at the same mu
        oref = orc.solve(sysm, mu, plan=po)
        err_o = max(float(np.max(np.abs(Dc_h[c_off[J]:c_off[J + 1]].reshape(-1, int(po.nbf[J])) -
                                        oref.subs[J].D_cols))) for J in range(n_mol))
        tS_o = np.array([oref.subs[J].t_S for J in range(n_mol)])
        print(f"mu={mu}: no-alloc vs solve_batch max|dD| = {err:.3e}, vs the FP64 oracle {err_o:.3e}")
        assert err <= TOL_D
        assert err_o <= TOL_D
        np.testing.assert_allclose(tS.cpu().numpy(), tS_o, rtol=TOL_TR, atol=TOL_TR)
        np.testing.assert_allclose(tS.cpu().numpy(), ref.sub_t_S.cpu().numpy(), rtol=TOL_TR, atol=TOL_TR)
        np.testing.assert_allclose(tH.cpu().numpy(), ref.sub_t_H.cpu().numpy(), rtol=TOL_TR, atol=TOL_TR)


def test_noalloc_rejects_oversized_submatrices():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_08245_gb300 as nl
    lib = nl._abi.load()
    dev = torch.device("cuda")
    one = torch.ones(1, dtype=torch.int32, device=dev)
    big = torch.full((1,), 193, dtype=torch.int32, device=dev)
    z64 = torch.zeros(1, dtype=torch.int64, device=dev)
    f = torch.zeros(1, dtype=torch.float32, device=dev)
    d = torch.zeros(2, dtype=torch.float64, device=dev)
    i = torch.zeros(1, dtype=torch.int32, device=dev)
    opts = nl.options("bf16x3")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.nolsm_sign_noalloc(1, big.data_ptr(), one.data_ptr(), z64.data_ptr(), z64.data_ptr(), f.data_ptr(),
                                d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), 0.0, ctypes.byref(opts), s,
                                d.data_ptr(), d.data_ptr(), d.data_ptr(), i.data_ptr(), i.data_ptr())
    assert rc == nl._abi.ERR_UNSUPPORTED
    assert b"192" in lib.nolsm_last_error()
    rc = lib.nolsm_sign_noalloc(5000, one.data_ptr(), one.data_ptr(), z64.data_ptr(), z64.data_ptr(), f.data_ptr(),
                                d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), 0.0, ctypes.byref(opts), s,
                                d.data_ptr(), d.data_ptr(), d.data_ptr(), i.data_ptr(), i.data_ptr())
    assert rc == nl._abi.ERR_UNSUPPORTED
    # E4M3 products need the symmetric form, which the no-alloc entry does not prepare
    opts8 = nl.options("fp8e4m3")
    rc = lib.nolsm_sign_noalloc(1, one.data_ptr(), one.data_ptr(), z64.data_ptr(), z64.data_ptr(), f.data_ptr(),
                                d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), 0.0, ctypes.byref(opts8), s,
                                d.data_ptr(), d.data_ptr(), d.data_ptr(), i.data_ptr(), i.data_ptr())
    assert rc == nl._abi.ERR_UNSUPPORTED
