"""The C-ABI library builds, loads without a GPU and exports every function include/nolsm.h declares;
the binding's ctypes structures match the header's layout. No compute calls (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(nolsm_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2104_08245_gb300 import _abi, build
    build.build()
    return _abi.load()


def test_header_declares_the_four_calls():
    names = header_functions()
    for n in ("nolsm_build_submatrices", "nolsm_solve_batch", "nolsm_scatter_density", "nolsm_find_mu"):
        assert n in names


def test_library_exports_every_declared_function(lib):
    from paper_2104_08245_gb300 import _abi
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.lib_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = header_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    bound = {n for n, _, _ in _abi.SIGNATURES}
    assert header_functions() == bound


def test_options_default_and_status_strings(lib):
    from paper_2104_08245_gb300 import _abi
    o = _abi.NolsmOptions()
    lib.nolsm_options_default(ctypes.byref(o), _abi.FP64)
    assert o.precision == _abi.FP64 and o.tol_ns == 1e-9 and o.max_iter == 100 and o.sub_end == 0
    lib.nolsm_options_default(ctypes.byref(o), _abi.FP8E4M3)
    assert o.refine_steps == 3
    assert lib.nolsm_status_str(_abi.ERR_NOT_SPD).decode().startswith("overlap")


def test_struct_layouts_match_header(tmp_path):
    """ctypes offsets and sizes equal those the C compiler gives for the header's structs."""
    from paper_2104_08245_gb300 import _abi
    structs = {"nolsm_system": _abi.NolsmSystem, "nolsm_options": _abi.NolsmOptions,
               "nolsm_plan_info": _abi.NolsmPlanInfo, "nolsm_stats": _abi.NolsmStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "nolsm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, got):
        cname, field, val = line.split()
        py = structs[cname]
        want = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert int(val) == want, (cname, field)


def test_null_arguments_are_rejected_without_a_gpu(lib):
    from paper_2104_08245_gb300 import _abi
    out = ctypes.c_void_p()
    assert lib.nolsm_build_submatrices(None, None, ctypes.byref(out)) == _abi.ERR_ARG
    assert lib.nolsm_scatter_density(None, None, None) == _abi.ERR_ARG
    assert b"NULL" in lib.nolsm_last_error() or lib.nolsm_last_error()


C_PROGRAM = r"""
#include <stdio.h>
#include "nolsm.h"
int main(void) {
  nolsm_options o;
  nolsm_options_default(&o, NOLSM_BF16X3);
  if (o.precision != NOLSM_BF16X3 || o.refine_steps != 2) return 1;
  nolsm_plan* plan = 0;
  if (nolsm_build_submatrices(0, 0, &plan) != NOLSM_ERR_ARG) return 2;
  /* the three-molecule chain: N(0) = {0,1}, N(1) = {0,1,2}, N(2) = {1,2}, one function each */
  int32_t nbf[3] = {1, 1, 1}, ptr[4] = {0, 2, 5, 7}, idx[7] = {0, 1, 0, 1, 2, 1, 2};
  int32_t group_of[3], ng = 0, sweeps = 0;
  double m[4];
  if (nolsm_combine_submatrices(3, nbf, ptr, idx, 1, group_of, &ng, m, &sweeps) != NOLSM_OK) return 3;
  printf("%d %d %d %d %d %.0f %.0f\n", group_of[0], group_of[1], group_of[2], ng, sweeps, m[0], m[1]);
  idx[0] = 1; idx[1] = 0;   /* N(0) no longer ascending */
  if (nolsm_combine_submatrices(3, nbf, ptr, idx, 1, group_of, &ng, m, &sweeps) != NOLSM_ERR_ARG) return 4;
  printf("%s\n", nolsm_status_str(NOLSM_ERR_ARG));
  return 0;
}
"""


def test_c_program_links_and_calls_the_host_entry_points(lib, tmp_path):
    """A C program built against include/nolsm.h and linked to the library calls the entry points
    that need no GPU (options, argument checks, the host-side combination heuristic)."""
    from paper_2104_08245_gb300 import _abi
    src = tmp_path / "host_calls.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "host_calls"
    libdir = os.path.dirname(_abi.lib_path())
    name = os.path.basename(_abi.lib_path())[3:-3]          # libnolsm.so -> nolsm
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, f"-l{name}",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, run.stdout + run.stderr
    first, second = run.stdout.splitlines()[:2]
    assert first == "0 0 0 1 3 43 27"
    assert second


def test_tuner_reports_no_shape_before_any_solve(lib):
    # the launch-shape tuner measures on the GPU at the first solve of a (kernel, precision, bucket); until then,
    # and for arguments out of range, it reports -1
    for kernel in (0, 1):
        for precision in range(6):
            for bucket in (0, 1):
                assert lib.nolsm_tc_shape(kernel, precision, bucket) == -1
    assert lib.nolsm_tc_shape(2, 1, 0) == -1
    assert lib.nolsm_tc_shape(0, 1, 2) == -1
    assert lib.nolsm_tc_shape(-1, 1, 0) == -1
