"""Python binding of the GB300 NOLSM library (include/nolsm.h).

The binding only marshals arguments: PyTorch supplies device memory and the stream, and every step of
the method runs in the library's CUDA kernels. Names follow the C ABI: ``nolsm_build_submatrices``,
``nolsm_solve_batch``, ``nolsm_scatter_density``, ``nolsm_find_mu``. There is no CPU fallback; the
library must be built (``__graft_entry__.build()``) and a CUDA device must be present.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

from . import _abi
from ._abi import (BF16, BF16X3, BOUND_GERSHGORIN, BOUND_MLP, BOUND_POWER, FP8E4M3, FP16, FP32, FP64,  # noqa: F401
                   PRECISIONS, NolsmOptions, NolsmPlanInfo, NolsmStats, NolsmSystem)

__all__ = ["DeviceSystem", "nolsm_build_submatrices", "nolsm_solve_batch", "nolsm_scatter_density",
           "nolsm_energy_weighted", "nolsm_combine_submatrices",
           "nolsm_find_mu", "nolsm_plan_query", "nolsm_plan_get_maps", "nolsm_plan_stats", "nolsm_plan_stats_reset",
           "nolsm_spectral_bracket", "nolsm_plan_get_prepared", "nolsm_plan_set_elements", "ElementModel", "nolsm_build_grouped",
           "nolsm_features", "nolsm_power_bounds", "nolsm_training_data",
           "nolsm_plan_set_mlp", "Mlp", "MLP_PARAMS",
           "options", "NolsmError", "Plan", "SolveResult", "MuResult"]


class NolsmError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _abi.load()
        msg = lib.nolsm_last_error().decode()
        super().__init__(f"{where}: {lib.nolsm_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def _torch():
    import torch
    return torch


def _stream(stream) -> ctypes.c_void_p:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def options(precision="fp64", **kw) -> NolsmOptions:
    """Default options of a precision (name or nolsm_precision value), then keyword overrides."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o = NolsmOptions()
    _abi.load().nolsm_options_default(ctypes.byref(o), p)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def nolsm_tc_shape(kernel: str, precision, bucket: int) -> int:
    """Launch shape chosen in this process (0 or 1, -1 while not measured) for kernel "sign" or "inverse",
    a precision (name or value; the inverse square root always runs in "fp16") and bucket 0 (n <= 192) or
    1 (n > 192)."""
    k = {"sign": 0, "inverse": 1}[kernel]
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return int(_abi.load().nolsm_tc_shape(k, p, int(bucket)))


class DeviceSystem:
    """Block-CSR S and H0 copied to device tensors (caller-owned memory for the ABI). values=False copies
    the patterns only (the elements are then generated on the device, nolsm_plan_set_elements)."""

    def __init__(self, system, device="cuda", values=True):
        torch = _torch()
        dev = torch.device(device)
        as_t = lambda a, dt: torch.as_tensor(a, dtype=dt).to(dev)
        self.n_mol = int(system.nbf.shape[0])
        self.nbf = as_t(system.nbf, torch.int32)
        self.s_row_ptr = as_t(system.S.row_ptr, torch.int32)
        self.s_col_idx = as_t(system.S.col_idx, torch.int32)
        self.s_vals = as_t(system.S.vals, torch.float64) if values else None
        self.h_row_ptr = as_t(system.H.row_ptr, torch.int32)
        self.h_col_idx = as_t(system.H.col_idx, torch.int32)
        self.h_vals = as_t(system.H.vals, torch.float64) if values else None
        self.n_occ = float(system.n_occ)

    def struct(self) -> NolsmSystem:
        s = NolsmSystem()
        s.n_mol = self.n_mol
        s.nbf = self.nbf.data_ptr()
        s.s_nnzb = self.s_col_idx.numel()
        s.s_row_ptr, s.s_col_idx, s.s_vals = (self.s_row_ptr.data_ptr(), self.s_col_idx.data_ptr(),
                                              _ptr(self.s_vals))
        s.h_nnzb = self.h_col_idx.numel()
        s.h_row_ptr, s.h_col_idx, s.h_vals = (self.h_row_ptr.data_ptr(), self.h_col_idx.data_ptr(),
                                              _ptr(self.h_vals))
        return s


def nolsm_build_submatrices(dsys: DeviceSystem, stream=None) -> "Plan":
    lib = _abi.load()
    st = dsys.struct()
    out = ctypes.c_void_p()
    rc = lib.nolsm_build_submatrices(ctypes.byref(st), _stream(stream), ctypes.byref(out))
    if rc != 0:
        raise NolsmError(rc, "nolsm_build_submatrices")
    return Plan(out, dsys)


class ElementModel:
    """Device copies of the geometry and the parameters of the synthetic element model for
    nolsm_plan_set_elements: positions [n_mol][3], the cell, every molecule's on-site energies in order, the
    S and H0 parameters and (for the direction modulation) the direction vectors [2][64][3]."""

    def __init__(self, system, device="cuda"):
        import numpy as np
        torch = _torch()
        dev = torch.device(device)
        sp = system.spec
        self.pos = torch.as_tensor(np.ascontiguousarray(system.pos), dtype=torch.float64).to(dev)
        self.onsite = torch.as_tensor(np.concatenate([np.asarray(o, dtype=np.float64) for o in system.onsite]),
                                      dtype=torch.float64).to(dev)
        dirs = np.zeros((2, 64, 3))
        if system.dirs is not None:
            dirs[:, :system.dirs.shape[1], :] = system.dirs
        self.dirs = torch.as_tensor(dirs, dtype=torch.float64).to(dev)
        self.cell = [float(c) for c in system.cell]
        self.params = (sp.s_exp, sp.hop, sp.hop_len, sp.aniso)

    def struct(self):
        m = _abi.NolsmElementModel()
        m.pos, m.onsite, m.dirs = self.pos.data_ptr(), self.onsite.data_ptr(), self.dirs.data_ptr()
        for k in range(3):
            m.cell[k] = self.cell[k]
        m.s_exp, m.hop, m.hop_len, m.aniso = self.params
        return m


def nolsm_plan_set_elements(plan: "Plan", model: ElementModel) -> None:
    """Generate the plan's matrix elements on the device from the geometry from now on."""
    m = model.struct()
    rc = _abi.load().nolsm_plan_set_elements(plan.handle, ctypes.byref(m))
    if rc != 0:
        raise NolsmError(rc, "nolsm_plan_set_elements")
    plan.model = model   # keeps the device arrays alive while the plan may use them


def nolsm_build_grouped(plan: "Plan", group_of, stream=None) -> "Plan":
    """A plan whose submatrices are the groups of molecules given by group_of (one label per molecule, e.g.
    nolsm_combine_submatrices(...).group_of)."""
    import numpy as np
    g = np.ascontiguousarray(np.asarray(group_of.cpu() if hasattr(group_of, "cpu") else group_of), dtype=np.int32)
    out = ctypes.c_void_p()
    rc = _abi.load().nolsm_build_grouped(plan.handle, g.ctypes.data, _stream(stream), ctypes.byref(out))
    if rc != 0:
        raise NolsmError(rc, "nolsm_build_grouped")
    gp = Plan(out, plan.dsys)
    gp.model = getattr(plan, "model", None)
    return gp


def nolsm_plan_query(plan: "Plan") -> NolsmPlanInfo:
    info = NolsmPlanInfo()
    rc = _abi.load().nolsm_plan_query(plan.handle, ctypes.byref(info))
    if rc != 0:
        raise NolsmError(rc, "nolsm_plan_query")
    return info


def nolsm_plan_get_maps(plan: "Plan", stream=None) -> dict:
    torch = _torch()
    info = nolsm_plan_query(plan)
    n, m, q = info.n_mol, info.d_nnzb, info.nb_entries
    dev = plan.dsys.nbf.device
    out = {"nb_ptr": torch.empty(n + 1, dtype=torch.int32, device=dev),
           "nb_idx": torch.empty(q, dtype=torch.int32, device=dev),
           "nb_off": torch.empty(q, dtype=torch.int32, device=dev),
           "sub_n": torch.empty(n, dtype=torch.int32, device=dev),
           "sub_c0": torch.empty(n, dtype=torch.int32, device=dev),
           "d_blk_off": torch.empty(m + 1, dtype=torch.int64, device=dev)}
    rc = _abi.load().nolsm_plan_get_maps(plan.handle, *(out[k].data_ptr() for k in
                                                        ("nb_ptr", "nb_idx", "nb_off", "sub_n", "sub_c0",
                                                         "d_blk_off")), _stream(stream))
    if rc != 0:
        raise NolsmError(rc, "nolsm_plan_get_maps")
    return out


def nolsm_plan_get_prepared(plan: "Plan", opts: NolsmOptions, stream=None):
    """(A, Q, prep_status, cond_est) device tensors of the options' preparation: A_J (float32, float64 for
    FP64) packed at the exclusive prefix sums of n_J^2, Q (float64, centre columns of T_J(S)^-1) at those of
    n_J b_J, and the preparation's lower estimate of cond(T_J(S)) (tensor-core standard form; else zero)."""
    torch = _torch()
    maps = nolsm_plan_get_maps(plan, stream)
    n = maps["sub_n"].to(torch.int64)
    b = plan.dsys.nbf.to(torch.int64)
    dev = plan.dsys.nbf.device
    A = torch.zeros(int((n * n).sum()), dtype=torch.float64 if opts.precision == FP64 else torch.float32, device=dev)
    Q = torch.zeros(int((n * b).sum()), dtype=torch.float64, device=dev)
    ps = torch.zeros(plan.dsys.n_mol, dtype=torch.int32, device=dev)
    rr = torch.zeros(plan.dsys.n_mol, dtype=torch.float32, device=dev)
    rc = _abi.load().nolsm_plan_get_prepared(plan.handle, ctypes.byref(opts), _stream(stream), A.data_ptr(),
                                             Q.data_ptr(), ps.data_ptr(), rr.data_ptr())
    if rc != 0:
        raise NolsmError(rc, "nolsm_plan_get_prepared")
    return A, Q, ps, rr


def nolsm_spectral_bracket(plan: "Plan", opts: NolsmOptions, stream=None):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    rc = _abi.load().nolsm_spectral_bracket(plan.handle, ctypes.byref(opts), _stream(stream), ctypes.byref(lo),
                                            ctypes.byref(hi))
    if rc != 0:
        raise NolsmError(rc, "nolsm_spectral_bracket")
    return lo.value, hi.value


def nolsm_bisect_begin(plan: "Plan", opts: NolsmOptions, bracket_contains_spectrum: bool, stream=None) -> None:
    rc = _abi.load().nolsm_bisect_begin(plan.handle, ctypes.byref(opts), _stream(stream),
                                        1 if bracket_contains_spectrum else 0)
    if rc != 0:
        raise NolsmError(rc, "nolsm_bisect_begin")


def nolsm_bisect_point(plan: "Plan", mu: float, opts: NolsmOptions, stream=None, check: bool = True):
    """One bisection point: (status, Tr(DS) over the options' range, submatrices solved)."""
    t, solved = ctypes.c_double(), ctypes.c_int32()
    rc = _abi.load().nolsm_bisect_point(plan.handle, float(mu), ctypes.byref(opts), _stream(stream),
                                        ctypes.byref(t), ctypes.byref(solved))
    if rc in (_abi.ERR_ARG, _abi.ERR_CUDA, _abi.ERR_OOM, _abi.ERR_UNSUPPORTED) or (check and rc != 0):
        raise NolsmError(rc, "nolsm_bisect_point")
    return rc, t.value, solved.value


def nolsm_bisect_side(plan: "Plan", opts: NolsmOptions, raises_lo: bool, stream=None) -> None:
    rc = _abi.load().nolsm_bisect_side(plan.handle, ctypes.byref(opts), _stream(stream), 1 if raises_lo else 0)
    if rc != 0:
        raise NolsmError(rc, "nolsm_bisect_side")


def nolsm_plan_stats(plan: "Plan") -> dict:
    st = NolsmStats()
    rc = _abi.load().nolsm_plan_stats(plan.handle, ctypes.byref(st))
    if rc != 0:
        raise NolsmError(rc, "nolsm_plan_stats")
    return st.as_dict()


def nolsm_plan_stats_reset(plan: "Plan") -> None:
    rc = _abi.load().nolsm_plan_stats_reset(plan.handle)
    if rc != 0:
        raise NolsmError(rc, "nolsm_plan_stats_reset")


@dataclasses.dataclass
class SolveResult:
    status: int
    trace_DS: float
    trace_DH: float
    sub_t_S: object = None
    sub_t_H: object = None
    iters: object = None
    sub_status: object = None


def nolsm_solve_batch(plan: "Plan", mu: float, opts: NolsmOptions, stream=None, per_sub: bool = True,
                      check: bool = True) -> SolveResult:
    """Solves every submatrix of the options' range at chemical potential mu. Raises on argument,
    CUDA or memory errors; per-submatrix outcomes are in ``status``/``sub_status`` (and raise only
    when ``check``)."""
    torch = _torch()
    lib = _abi.load()
    n = plan.dsys.n_mol
    dev = plan.dsys.nbf.device
    tS, tH = ctypes.c_double(), ctypes.c_double()
    sts = sth = it = sst = None
    if per_sub:
        sts = torch.zeros(n, dtype=torch.float64, device=dev)
        sth = torch.zeros(n, dtype=torch.float64, device=dev)
        it = torch.zeros(n, dtype=torch.int32, device=dev)
        sst = torch.zeros(n, dtype=torch.int32, device=dev)
    rc = lib.nolsm_solve_batch(plan.handle, float(mu), ctypes.byref(opts), _stream(stream), ctypes.byref(tS),
                               ctypes.byref(tH), _ptr(sts), _ptr(sth), _ptr(it), _ptr(sst))
    if rc in (_abi.ERR_ARG, _abi.ERR_CUDA, _abi.ERR_OOM, _abi.ERR_UNSUPPORTED) or (check and rc != 0):
        raise NolsmError(rc, "nolsm_solve_batch")
    return SolveResult(rc, tS.value, tH.value, sts, sth, it, sst)


def nolsm_scatter_density(plan: "Plan", D_vals=None, stream=None):
    torch = _torch()
    if D_vals is None:
        D_vals = torch.zeros(nolsm_plan_query(plan).d_nvals, dtype=torch.float64, device=plan.dsys.nbf.device)
    rc = _abi.load().nolsm_scatter_density(plan.handle, D_vals.data_ptr(), _stream(stream))
    if rc != 0:
        raise NolsmError(rc, "nolsm_scatter_density")
    return D_vals


def nolsm_energy_weighted(plan: "Plan", W_vals=None, stream=None):
    """(W in the merged pattern of D, sum of the T_J(W) T_J(S) partial traces) at the plan's solution;
    W_vals=False skips the write-back (trace only)."""
    torch = _torch()
    if W_vals is None:
        W_vals = torch.zeros(nolsm_plan_query(plan).d_nvals, dtype=torch.float64, device=plan.dsys.nbf.device)
    tw = ctypes.c_double()
    rc = _abi.load().nolsm_energy_weighted(plan.handle, _stream(stream), W_vals.data_ptr() if W_vals is not False
                                           else None, ctypes.byref(tw))
    if rc != 0:
        raise NolsmError(rc, "nolsm_energy_weighted")
    return (W_vals if W_vals is not False else None), tw.value


@dataclasses.dataclass
class CombineResult:
    group_of: "np.ndarray"    # int32 [n_mol]: each molecule's group (its smallest member)
    n_groups: int
    sum_n3_before: float
    sum_n3_after: float
    sum_n2_before: float
    sum_n2_after: float
    sweeps: int


def nolsm_combine_submatrices(nbf, nb_ptr, nb_idx, threads: int = 0) -> CombineResult:
    """Submatrix combination heuristic on a host copy of the merged pattern (numpy arrays or CPU tensors)."""
    import numpy as np
    a = [np.ascontiguousarray(np.asarray(x.cpu() if hasattr(x, "cpu") else x), dtype=np.int32)
         for x in (nbf, nb_ptr, nb_idx)]
    n_mol = int(a[0].shape[0])
    group_of = np.zeros(n_mol, dtype=np.int32)
    metrics = np.zeros(4, dtype=np.float64)
    ng, sw = ctypes.c_int32(), ctypes.c_int32()
    rc = _abi.load().nolsm_combine_submatrices(n_mol, a[0].ctypes.data, a[1].ctypes.data, a[2].ctypes.data,
                                               int(threads), group_of.ctypes.data, ctypes.byref(ng),
                                               metrics.ctypes.data, ctypes.byref(sw))
    if rc != 0:
        raise NolsmError(rc, "nolsm_combine_submatrices")
    return CombineResult(group_of, ng.value, *[float(x) for x in metrics], sw.value)


@dataclasses.dataclass
class MuResult:
    status: int
    mu: float
    trace_DS: float
    steps: int
    history: list


def nolsm_find_mu(plan: "Plan", n_occ: float, lo: float, hi: float, opts: NolsmOptions, stream=None,
                  check: bool = False) -> MuResult:
    lib = _abi.load()
    mu, t, steps = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    cap = opts.max_bisect if opts.max_bisect > 0 else 100
    hist = (ctypes.c_double * cap)()
    rc = lib.nolsm_find_mu(plan.handle, float(n_occ), float(lo), float(hi), ctypes.byref(opts), _stream(stream),
                           ctypes.byref(mu), ctypes.byref(t), ctypes.byref(steps), hist)
    if rc in (_abi.ERR_ARG, _abi.ERR_CUDA, _abi.ERR_OOM, _abi.ERR_UNSUPPORTED) or (check and rc != 0):
        raise NolsmError(rc, "nolsm_find_mu")
    return MuResult(rc, mu.value, t.value, steps.value, list(hist[:steps.value]))


class Plan:
    """Owner of a nolsm_plan handle (destroyed with the object or by ``close``)."""

    def __init__(self, handle: ctypes.c_void_p, dsys: DeviceSystem):
        self.handle = handle
        self.dsys = dsys      # keeps the caller-owned input tensors alive

    def close(self):
        if self.handle is not None and self.handle.value:
            _abi.load().nolsm_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # conveniences with the same semantics as the module functions
    def info(self):
        return nolsm_plan_query(self)

    def maps(self, stream=None):
        return nolsm_plan_get_maps(self, stream)

    def solve(self, mu, opts, **kw):
        return nolsm_solve_batch(self, mu, opts, **kw)

    def scatter(self, D_vals=None, stream=None):
        return nolsm_scatter_density(self, D_vals, stream)

    def find_mu(self, n_occ, lo, hi, opts, **kw):
        return nolsm_find_mu(self, n_occ, lo, hi, opts, **kw)

    def energy_weighted(self, W_vals=None, stream=None):
        return nolsm_energy_weighted(self, W_vals, stream)

    def stats(self):
        return nolsm_plan_stats(self)

    def stats_reset(self):
        nolsm_plan_stats_reset(self)


# ------------------------------------------------------------------------------------ a4 bounds, a10 network

def nolsm_features(plan: "Plan", mu: float, opts: NolsmOptions, stream=None):
    """float32 [n_mol, 7] device tensor of features (rows of the options' range written)."""
    torch = _torch()
    feat = torch.zeros(plan.dsys.n_mol, 7, dtype=torch.float32, device=plan.dsys.nbf.device)
    rc = _abi.load().nolsm_features(plan.handle, float(mu), ctypes.byref(opts), _stream(stream), feat.data_ptr())
    if rc != 0:
        raise NolsmError(rc, "nolsm_features")
    return feat


def nolsm_power_bounds(plan: "Plan", opts: NolsmOptions, stream=None):
    """float64 [n_mol, 2] device tensor of power-iteration intervals (rows of the options' range written)."""
    torch = _torch()
    lam = torch.zeros(plan.dsys.n_mol, 2, dtype=torch.float64, device=plan.dsys.nbf.device)
    rc = _abi.load().nolsm_power_bounds(plan.handle, ctypes.byref(opts), _stream(stream), lam.data_ptr())
    if rc != 0:
        raise NolsmError(rc, "nolsm_power_bounds")
    return lam


def nolsm_training_data(plan: "Plan", mu: float, opts: NolsmOptions, stream=None):
    """(x [n_mol, 7], t [n_mol, 3]) float32 device tensors: features and the method's own targets."""
    torch = _torch()
    dev = plan.dsys.nbf.device
    x = torch.zeros(plan.dsys.n_mol, 7, dtype=torch.float32, device=dev)
    t = torch.zeros(plan.dsys.n_mol, 3, dtype=torch.float32, device=dev)
    rc = _abi.load().nolsm_training_data(plan.handle, float(mu), ctypes.byref(opts), _stream(stream), x.data_ptr(),
                                         t.data_ptr())
    if rc != 0:
        raise NolsmError(rc, "nolsm_training_data")
    return x, t


def nolsm_plan_set_mlp(plan: "Plan", mlp: Optional["Mlp"]) -> None:
    rc = _abi.load().nolsm_plan_set_mlp(plan.handle, None if mlp is None else mlp.handle)
    if rc != 0:
        raise NolsmError(rc, "nolsm_plan_set_mlp")
    plan.mlp = mlp   # keeps the network alive while the plan may use it


MLP_PARAMS = 17923


class Mlp:
    """Owner of a nolsm_mlp handle: the learned bound predictor's network (FP32 on the device)."""

    def __init__(self, seed: int = 0, stream=None):
        lib = _abi.load()
        h = ctypes.c_void_p()
        rc = lib.nolsm_mlp_create(ctypes.c_uint64(seed), _stream(stream), ctypes.byref(h))
        if rc != 0:
            raise NolsmError(rc, "nolsm_mlp_create")
        self.handle = h
        self.n_params = lib.nolsm_mlp_param_count()

    def close(self):
        if self.handle is not None and self.handle.value:
            _abi.load().nolsm_mlp_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import numpy as np
        out = np.zeros(self.n_params, dtype=np.float32)
        rc = _abi.load().nolsm_mlp_get_params(self.handle, out.ctypes.data)
        if rc != 0:
            raise NolsmError(rc, "nolsm_mlp_get_params")
        return out

    def set_params(self, params) -> None:
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.size}")
        rc = _abi.load().nolsm_mlp_set_params(self.handle, p.ctypes.data)
        if rc != 0:
            raise NolsmError(rc, "nolsm_mlp_set_params")

    def forward(self, x, stream=None):
        torch = _torch()
        x = x.contiguous()
        y = torch.zeros(x.shape[0], 3, dtype=torch.float32, device=x.device)
        rc = _abi.load().nolsm_mlp_forward(self.handle, int(x.shape[0]), x.data_ptr(), y.data_ptr(), _stream(stream))
        if rc != 0:
            raise NolsmError(rc, "nolsm_mlp_forward")
        return y

    def gradient(self, x, t, stream=None):
        """(flat float32 gradient on the host, loss) of the batch."""
        import numpy as np
        x, t = x.contiguous(), t.contiguous()
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        rc = _abi.load().nolsm_mlp_gradient(self.handle, int(x.shape[0]), x.data_ptr(), t.data_ptr(),
                                            _stream(stream), g.ctypes.data, ctypes.byref(loss))
        if rc != 0:
            raise NolsmError(rc, "nolsm_mlp_gradient")
        return g, loss.value

    def adam_step(self, lr: float, stream=None) -> None:
        rc = _abi.load().nolsm_mlp_adam_step(self.handle, ctypes.c_float(lr), _stream(stream))
        if rc != 0:
            raise NolsmError(rc, "nolsm_mlp_adam_step")

    def train(self, x, t, epochs: int, batch: int, lr: float, stream=None):
        """Per-epoch mean minibatch loss (list)."""
        x, t = x.contiguous(), t.contiguous()
        losses = (ctypes.c_double * epochs)()
        rc = _abi.load().nolsm_mlp_train(self.handle, int(x.shape[0]), x.data_ptr(), t.data_ptr(), int(epochs),
                                         int(batch), ctypes.c_float(lr), _stream(stream), losses)
        if rc != 0:
            raise NolsmError(rc, "nolsm_mlp_train")
        return list(losses)
