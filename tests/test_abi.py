"""CPU checks of the C ABI boundary: the library builds, loads, exports every
function include/pdqp.h declares, and the ctypes structs match the C layout.
No compute call is made (there may be no GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdqp.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def _declared_functions(path):
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pdqp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_07710_gb300 import build, pdqp
    build.build()
    return pdqp.load()


def test_header_declares_the_boundary():
    names = _declared_functions(HEADER)
    for required in ("pdqp_create", "pdqp_solve", "pdqp_solve_batch", "pdqp_destroy", "pdqp_default_options"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2311_07710_gb300 import pdqp
    assert len(HEADERS) >= 2
    for name in sorted({n for h in HEADERS for n in _declared_functions(h)}):
        assert hasattr(lib, name), name
        assert name in pdqp.SIGNATURES, f"binding lacks {name}"


def test_struct_layout_matches_c(tmp_path, lib):
    from paper_2311_07710_gb300 import pdqp
    import ctypes
    fields = {"pdqp_options": [f for f, _ in pdqp.pdqp_options._fields_], "pdqp_profile": [f for f, _ in pdqp.pdqp_profile._fields_],
              "pdqp_info": [f for f, _ in pdqp.pdqp_info._fields_],
              "pdqp_ws_train_options": [f for f, _ in pdqp.pdqp_ws_train_options._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>'] + [f'#include "{h}"' for h in HEADERS] + ["int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", str(src), "-o", str(exe)])
    out = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)]).decode().split("\n") if line)
    for st, fs in fields.items():
        cls = getattr(pdqp, st)
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fs:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, f"{st}.{f}"


def test_default_options_and_status_strings(lib):
    from paper_2311_07710_gb300 import pdqp
    o = pdqp.pdqp_default_options()
    assert (o.ruiz_iters, o.check_period, o.max_iter) == (10, 64, 200000)
    assert (o.beta_suff, o.beta_nec, o.beta_art, o.pw_theta) == (0.2, 0.8, 0.36, 0.2)
    assert o.eps == 1e-6 and o.eps_zero == 1e-10
    assert pdqp.status_string(pdqp.PDQP_OK) == "optimal"
    assert pdqp.status_string(pdqp.PDQP_ITER_LIMIT) == "iteration limit"


def test_invalid_input_is_rejected_on_the_host(lib):
    """Validation runs before any device work, so it is checkable here; the
    first CUDA call may fail without a GPU, which also must not crash."""
    import numpy as np
    from paper_2311_07710_gb300 import pdqp
    rp = np.array([0, 1, 2], np.int32)
    bad_col = np.array([0, 5], np.int32)         # column out of range
    v = np.ones(2)
    with pytest.raises(pdqp.PdqpError) as e:
        pdqp.pdqp_create(2, 0, 0, rp, bad_col, v, np.zeros(1, np.int32), None, None, np.zeros(2), None,
                         -np.ones(2), np.ones(2))
    assert e.value.status in (pdqp.PDQP_ERR_INVALID, pdqp.PDQP_ERR_CUDA)
