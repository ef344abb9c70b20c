"""C-ABI checks that need no GPU: the library builds, loads, and exports
every function that include/lbib.h declares; the Python binding uses the
same names; a missing library is a loud error, never a fallback."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbib.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbib_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2207_06029_gb300 import build
    return build.build()


def test_header_declares_the_path_calls():
    names = _declared()
    for required in ["lbib_create", "lbib_add_body", "lbib_step", "lbib_get_fields", "lbib_get_markers",
                     "lbib_destroy", "lbib_last_error", "lbib_sync"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbib_[a-z_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_uses_the_same_names(libpath):
    from paper_2207_06029_gb300 import lbib
    L = lbib.load()
    for name in _declared():
        assert hasattr(L, name)
        assert hasattr(lbib, name), f"binding lacks {name}"


def test_missing_library_fails_loudly(tmp_path):
    code = ("import paper_2207_06029_gb300.lbib as m; m.LIB_PATH = '/nonexistent/liblbib.so'\n"
            "try:\n    m.load()\nexcept RuntimeError as e:\n    print('RAISED', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "RAISED" in r.stdout and "no CPU fallback" in r.stdout


def test_create_rejects_bad_parameters_without_touching_the_gpu(libpath):
    """Argument validation happens before any CUDA call."""
    from paper_2207_06029_gb300 import lbib
    for kw in [dict(n=(8, 8, 8), tau=0.5), dict(n=(0, 8, 8), tau=0.8), dict(n=(8, 8, 2), tau=0.8, bc=(0, 0, 1))]:
        p = lbib.make_params(kw["n"], kw["tau"], bc=kw.get("bc", (0, 0, 0)))
        with pytest.raises(lbib.LbibError) as ei:
            lbib.lbib_create(p)
        assert ei.value.code == lbib.LBIB_EINVAL
    p = lbib.make_params((8, 8, 8), 0.8, precision=7)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_create(p)


def test_serve_create_rejects_bad_parameters_without_touching_the_gpu(libpath):
    """Server parameters are checked before the worker, stream or device are
    touched: no budget, no active slot, an unknown mode or batch order."""
    from paper_2207_06029_gb300 import lbib
    for kw in [dict(hbm_budget=0), dict(hbm_budget=1 << 30, max_active=0), dict(hbm_budget=1 << 30, mode=2),
               dict(hbm_budget=1 << 30, batch_order=2), dict(hbm_budget=1 << 30, batch_order=-1)]:
        with pytest.raises(lbib.LbibError) as ei:
            lbib.lbib_serve_create(**kw)
        assert ei.value.code == lbib.LBIB_EINVAL, kw


def test_measure_fma_rejects_a_null_output_without_touching_the_gpu(libpath):
    from paper_2207_06029_gb300 import lbib
    import ctypes as C
    assert lbib.load().lbib_measure_fma(1, C.cast(None, C.POINTER(C.c_double))) == lbib.LBIB_EINVAL


@pytest.mark.gpu
def test_measured_fma_rates_are_positive_and_fp64_is_the_slower(libpath):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06029_gb300 import lbib
    f64, f32 = lbib.lbib_measure_fma(True), lbib.lbib_measure_fma(False)
    assert 0.0 < f64 < f32


STRUCTS = ["lbib_params", "lbib_body_params", "lbib_body_state", "lbib_serve_params", "lbib_serve_times",
           "lbib_serve_summary"]


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the header's field names,
    offsets and size, as gcc lays out include/lbib.h (a field added to the
    header but not to the binding would shift every later field)."""
    import ctypes
    from paper_2207_06029_gb300 import lbib as L
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbib.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(L, name)._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    want = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        want[(s, f)] = int(v)
    for name in STRUCTS:
        cls = getattr(L, name)
        assert ctypes.sizeof(cls) == want[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == want[(name, field)], (name, field)
