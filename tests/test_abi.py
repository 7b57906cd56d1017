"""Host-side checks of the C ABI: the library builds, loads, and exports every entry point
that include/bem.h declares. No GPU compute."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1905_01341_gb300 import build

    build.build()
    from paper_1905_01341_gb300 import bem

    return bem.lib()


def test_header_declares_the_boundary():
    names = set(_declared_functions())
    for required in ("bem_mesh_upload", "fmm_build", "bem_apply_sl", "bem_apply_dl", "bem_solve", "bem_create",
                     "bem_destroy", "bem_apply", "bem_rhs", "bem_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1905_01341_gb300 import bem

    for name in _declared_functions():
        assert name in bem.EXPORTED and callable(getattr(bem, name)), name


def test_params_default_host_only(lib):
    from paper_1905_01341_gb300 import bem

    p = bem.bem_params_default()
    assert p.p_fmm == 14 and p.precision == bem.BEM_PREC_MIXED and p.gmres_tol == 1e-6
    assert p.gmres_maxit == 100 and p.diag_precision == -1 and p.m2l_tensor_cores == 3
    p2 = bem.bem_params_default(p_fmm=16, precision=bem.BEM_PREC_FP64)
    assert p2.p_fmm == 16 and p2.precision == 0


def _c_layout(struct, fields):
    """sizeof and field offsets of a struct of include/bem.h, from a C program built with gcc."""
    import subprocess
    import tempfile

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    body = 'printf("%zu", sizeof(' + struct + '));' + "".join(
        'printf(" %zu", offsetof(' + struct + ', ' + f + '));' for f in fields)
    src = "#include <stddef.h>\n#include <stdio.h>\n#include \"bem.h\"\nint main(void) { " + body + " return 0; }\n"
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        with open(c, "w") as fh:
            fh.write(src)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(root, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(x) for x in out]


@pytest.mark.parametrize("name", ["bem_params", "bem_stats", "bem_step_params", "bem_step_stats"])
def test_struct_layouts_match_header(name):
    import ctypes

    from paper_1905_01341_gb300 import bem

    cls = getattr(bem, name)
    fields = [f for f, _ in cls._fields_]
    want = _c_layout(name, fields)
    got = [ctypes.sizeof(cls)] + [getattr(cls, f).offset for f in fields]
    assert got == want


def test_struct_defaults():
    from paper_1905_01341_gb300 import bem

    assert bem.bem_params_default().gmres_precond == 0
    assert bem.bem_params_default().overlap == 1 and bem.bem_params_default().diag_p_fmm == -1
    assert bem.bem_params_default().m2l_stages == 0 and bem.bem_params_default().p2p_blocks_per_sm == -1
    sp = bem.bem_step_params_default()
    assert sp.pf == 6 and sp.courant == 0.1 and sp.kappa == 1.4 and sp.guess == 2
    assert [bem.bem_phase_name(i) for i in range(bem.BEM_NUM_PHASES)][6] == "m2l"


def test_create_reports_errors_without_gpu(lib):
    import torch

    from paper_1905_01341_gb300 import bem

    if torch.cuda.is_available():
        pytest.skip("GPU present: covered by the GPU tests")
    with pytest.raises(bem.BemError):
        bem.bem_create(bem.bem_params_default(), 0)
