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
    lib.tc_probe_trim.restype = ctypes.c_int
    lib.tc_probe_trim.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 6 + [ctypes.c_void_p]
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


def run_trim(probe, K, Nl, M, N, Kuse, dt, seed=0):
    """The raw accumulator (128 lanes x Nl columns) of a three-term product of random operands trimmed to
    M x N x Kuse, and the FP64 product of the same rounded operands over the trimmed shape."""
    import torch
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(128, K, generator=g, dtype=torch.float64)
    B = torch.randn(K, Nl, generator=g, dtype=torch.float64)
    Ah, Al = split(A, dt)
    Bh, Bl = split(B, dt)
    a, b = slice(0, M), slice(0, Kuse)
    ref = (Ah[a, b].double() @ Bh[b, :N].double() + Ah[a, b].double() @ Bl[b, :N].double()
           + Al[a, b].double() @ Bh[b, :N].double())
    Ad = torch.stack([Ah, Al]).contiguous().view(torch.int16).cuda()
    Bd = torch.stack([Bh, Bl]).contiguous().view(torch.int16).cuda()
    C = torch.zeros(128, Nl, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = probe.tc_probe_trim(Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), K, Nl, M, N, Kuse,
                             1 if dt == torch.bfloat16 else 0, err.data_ptr())
    assert rc == 0 and int(err.item()) == 0
    return C.cpu().double(), ref


@pytest.mark.parametrize("N,Kuse", [(160, 160), (176, 176), (192, 160), (160, 192), (144, 144)])
def test_products_trimmed_to_16_columns_and_16_k(probe, N, Kuse):
    """An M = 128 product over the first Kuse of K = 192 and the first N of 192 loaded columns (multiples of
    16, not of the 64-column chunks): the operands' entries past Kuse and N (random here) do not enter, and
    the accumulator's first N columns hold the product."""
    import torch
    C, ref = run_trim(probe, 192, 192, 128, N, Kuse, torch.float16)
    e = float((C[:, :N] - ref).abs().max() / ref.abs().max())
    print(f"M 128, N {N}, K {Kuse} of 192: rel err {e:.2e}")
    assert e < 1e-5


def test_m64_accumulator_layout(probe):
    """Where an M = 64 product's rows land in tensor memory, read back with the 32x32b loads: row r of the
    product in lane 32 (r // 16) + r % 16 (the first 16 lanes of each warp's quarter), columns in place,
    every other lane untouched."""
    import torch
    C, ref = run_trim(probe, 192, 192, 64, 192, 192, torch.float16)
    scale = float(ref.abs().max())
    found = {}
    for r in range(64):
        d = (C - ref[r][None, :]).abs().max(dim=1).values / scale
        lanes = [int(l) for l in torch.nonzero(d < 1e-5).flatten()]
        found[r] = lanes
    print("M 64 rows -> lanes:", {r: found[r] for r in range(0, 64, 8)})
    want = {r: [32 * (r // 16) + r % 16] for r in range(64)}
    assert found == want
    used = set(l for v in want.values() for l in v)
    rest = [l for l in range(128) if l not in used]
    assert float(C[rest].abs().max()) == 0.0
