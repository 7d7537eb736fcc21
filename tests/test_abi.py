"""The C-ABI library builds, loads and exports every declared entry point (CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eigdc.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(eig_[A-Za-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_1011_3077_gb300 import build
    return build.build()


def test_header_declares_the_path():
    names = _declared()
    for must in ("eig_divide_step", "eig_split", "eig_solve", "eig_create", "eig_destroy",
                 "eig_qr", "eig_haar", "eig_split_test", "eig_gemm", "eig_split_pencil",
                 "eig_pencil_schur"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_covers_header(built):
    from paper_1011_3077_gb300 import eigdc
    assert set(_declared()) == set(eigdc.EXPORTED)
    eigdc.lib()


def test_default_params_host_only(built):
    from paper_1011_3077_gb300 import eigdc
    p = eigdc.default_params()
    assert p.maxit == 60 and p.split_tol == 0.0 and p.leaf_size == 64 and p.v_draws == 4
    assert p.workers == 8 and p.graphs == 0


def test_struct_layout_matches_c_compiler(built, tmp_path):
    """The ctypes mirrors have the sizes and offsets the C compiler gives."""
    import shutil
    import subprocess
    from paper_1011_3077_gb300 import eigdc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "eigdc.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(eig_params_t),'
        ' sizeof(eig_region_t), sizeof(eig_step_info_t), sizeof(eig_solve_info_t),'
        ' offsetof(eig_params_t, seed), offsetof(eig_params_t, root_unit_circle),'
        ' offsetof(eig_solve_info_t, flops), sizeof(eig_enclosure_t),'
        ' offsetof(eig_enclosure_t, nhp), offsetof(eig_enclosure_t, t)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(eigdc.Params), ctypes.sizeof(eigdc.Region),
            ctypes.sizeof(eigdc.StepInfo), ctypes.sizeof(eigdc.SolveInfo),
            eigdc.Params.seed.offset, eigdc.Params.root_unit_circle.offset,
            eigdc.SolveInfo.flops.offset, ctypes.sizeof(eigdc.Enclosure),
            eigdc.Enclosure.nhp.offset, eigdc.Enclosure.t.offset]
    assert got == want


def test_fail_allocation_switch(built):
    """The host-side fault-injection switch (no GPU work)."""
    from paper_1011_3077_gb300 import eigdc
    assert eigdc.eig_debug_fail_allocations(0) >= 0
    assert eigdc.eig_debug_fail_allocations(2) == 0
    assert eigdc.eig_debug_fail_allocations(0) == 2
    assert eigdc.eig_debug_fail_allocations(-1) == eigdc.EIG_ERR_ARG
    assert eigdc.eig_debug_fail_allocations(0) == 0
