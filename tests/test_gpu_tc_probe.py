"""Tensor-core building blocks in isolation: one CTA computes C[128 x N] = A[128 x K] B[K x N] through
TMA (128-byte swizzle), the K-major / MN-major shared-memory descriptors, tcgen05.mma (one product,
or the three-term hi/lo split) and tcgen05.ld. Compared with an FP64 product of the same rounded
operands (PyTorch CPU)."""
import ctypes
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    so = str(tmp_path_factory.mktemp("probe") / "tc_probe.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-shared", "-I", os.path.join(ROOT, "paper_2104_08245_gb300", "csrc"), "-I",
                    os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "cuda", "tc_probe.cu"), "-o", so],
                   check=True)
    lib = ctypes.CDLL(so)
    lib.tc_probe_gemm.restype = ctypes.c_int
    lib.tc_probe_gemm.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 7 + [ctypes.c_void_p]
    return lib


def split(x, dt):
    import torch
    hi = x.to(dt)
    lo = (x - hi.double()).to(dt)
    return hi, lo


def run(probe, K, N, terms, dt, b_mn, lbo, sbo, seed=0):
    import torch
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(128, K, generator=g, dtype=torch.float64)
    B = torch.randn(K, N, generator=g, dtype=torch.float64)
    Ah, Al = split(A, dt)
    Bh, Bl = split(B, dt)
    if terms == 1:
        ref = Ah.double() @ Bh.double()
        Ad = Ah.view(torch.int16)[None]
        Bd = (Bh if b_mn else Bh.T.contiguous()).view(torch.int16)[None]
    else:
        ref = Ah.double() @ Bh.double() + Ah.double() @ Bl.double() + Al.double() @ Bh.double()
        Ad = torch.stack([Ah, Al]).view(torch.int16)
        Bd = (torch.stack([Bh, Bl]) if b_mn else torch.stack([Bh.T, Bl.T])).contiguous().view(torch.int16)
    Ad, Bd = Ad.contiguous().cuda(), Bd.contiguous().cuda()
    C = torch.zeros(128, N, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = probe.tc_probe_gemm(Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), K, N, terms,
                             1 if dt == torch.bfloat16 else 0, b_mn, lbo, sbo, err.data_ptr())
    assert rc == 0 and int(err.item()) == 0
    got = C.cpu().double()
    return float((got - ref).abs().max() / ref.abs().max())


@pytest.mark.parametrize("N", [64, 128, 256])
@pytest.mark.parametrize("dtname", ["bf16", "fp16"])
def test_mma_k_major_b(probe, N, dtname):
    import torch
    dt = torch.bfloat16 if dtname == "bf16" else torch.float16
    assert run(probe, 128, N, 1, dt, 0, 16, 1024) < 1e-6


@pytest.mark.parametrize("N", [64, 128, 192, 256])
@pytest.mark.parametrize("dtname", ["bf16", "fp16"])
def test_mma_mn_major_b(probe, N, dtname):
    """B row-major (K rows, N contiguous): 64-column chunks 8 KB apart (leading byte offset), 8-row
    groups 1 KB apart (stride byte offset)."""
    import torch
    dt = torch.bfloat16 if dtname == "bf16" else torch.float16
    assert run(probe, 192, N, 1, dt, 1, 8192, 1024) < 1e-6


@pytest.mark.parametrize("dtname", ["bf16", "fp16"])
def test_three_term_split_accumulates(probe, dtname):
    import torch
    dt = torch.bfloat16 if dtname == "bf16" else torch.float16
    # FP32 accumulation over K = 256; a missing lo product would leave an error near 4e-3 (bf16)
    assert run(probe, 256, 256, 3, dt, 1, 8192, 1024) < 1e-5
