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
    assert bem.bem_params_default().overlap == -1 and bem.bem_params_default().diag_p_fmm == -1
    assert bem.bem_params_default().m2l_stages == 0 and bem.bem_params_default().p2p_blocks_per_sm == -1
    assert bem.bem_params_default().m2l_target_major == 1
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


def test_entry_points_reject_a_null_context():
    """Every entry point that takes a context returns BEM_ERR_ARG for a NULL one, with the reason
    in bem_last_error(NULL), before any CUDA call (host only): the context check comes first in
    each of them, the ones added for the preconditioner and the filter included."""
    import ctypes

    from paper_1905_01341_gb300 import bem

    L = bem.lib()
    checked = []
    for name in bem.EXPORTED:
        fn = getattr(L, name)
        args = fn.argtypes or []
        if not args or args[0] is not ctypes.c_void_p or fn.restype is not ctypes.c_int:
            continue
        vals = []
        for a in args:
            if a is ctypes.c_double:
                vals.append(0.0)
            elif a in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64):
                vals.append(0)
            else:
                vals.append(None)
        assert fn(*vals) == bem.BEM_ERR_ARG, name
        assert b"null context" in L.bem_last_error(None), name
        checked.append(name)
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "bem.h")).read(), flags=re.S)
    with_ctx = set(re.findall(r"^int\s+([a-z_0-9]+)\s*\(\s*void\s*\*\s*ctx\b", text, re.M))
    assert set(checked) == with_ctx
    assert {"bem_precond_apply", "bem_step_filter", "bem_solve"} <= with_ctx


def test_m2l_class_orders_follow_the_separation():
    """Per-class M2L truncation (host logic, no GPU): margin -1 keeps every class at p; otherwise
    the six nearest classes (face offsets 2 boxes apart) keep p, orders never grow with the
    distance of the offset, they are symmetric under sign flips and permutations of the axes
    (the ratio depends on |d| only), and they shrink towards the far corners but stay >= 1."""
    import math

    from paper_1905_01341_gb300 import bem

    offs = [(x, y, z) for x in range(-3, 4) for y in range(-3, 4) for z in range(-3, 4)
            if max(abs(x), abs(y), abs(z)) >= 2]
    assert len(offs) == 316
    assert bem.bem_m2l_orders(14, -1) == [14] * 316
    for p, margin in ((14, 6), (16, 6), (14, 0), (8, 2)):
        o = bem.bem_m2l_orders(p, margin)
        by = dict(zip(offs, o))
        for d in ((2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, 0, -2)):
            assert by[d] == p
        assert all(1 <= v <= p for v in o)
        dist = {d: math.sqrt(sum(c * c for c in d)) for d in offs}
        for d in offs:
            for e in offs:
                if dist[d] < dist[e] - 1e-12:
                    assert by[d] >= by[e]
            assert by[d] == by[tuple(-c for c in d)] == by[(d[1], d[2], d[0])]
        assert by[(3, 3, 3)] < p or margin >= p
    # more margin never lowers an order
    a, b = bem.bem_m2l_orders(14, 2), bem.bem_m2l_orders(14, 6)
    assert all(x <= y for x, y in zip(a, b))
