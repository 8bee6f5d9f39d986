"""Host-side checks of the C-ABI library (no GPU compute): it loads, exports
every function include/reg.h declares, and its scan schedules are the
oracle's, op for op."""
import ctypes
import os
import re
import subprocess

import pytest

from oracle import schedules as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1712_02533_gb300 import _build
    _build.build()
    import paper_1712_02533_gb300 as reg
    return reg


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(reg_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert {"reg_create_series", "reg_apply_operator_batch", "reg_prefix_scan", "reg_get_deformations"} <= declared
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared if not hasattr(so, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (reg_\w+)", out))
    assert declared <= exported


def test_status_strings_and_defaults(lib):
    so = lib._load()
    assert so.reg_status_string(0) == b"ok"
    assert b"invalid" in so.reg_status_string(1)
    p = lib.default_params()
    assert p.n_levels == 3 and p.iter_max == 50 and p.armijo_sigma == 0.5 and p.trials_per_pass == 4
    # every field after the first ones as well: the binding's struct layout is the header's
    assert p.epsilon == 1e-7 and p.lambda_ == 10.0 and p.tau_init == 1.0 and p.tau_max == 1e4
    assert p.tau_min == 1e-12 and p.storage == lib.STORAGE_F32 and p.max_steps == 0 and p.flags == 0
    assert p.init_levels == 0 and p.learned_fallback_px == 2.0
    assert not p.allocator.alloc and not p.allocator.free


def _norm(levels):
    return [sorted(lv) for lv in levels if lv]


@pytest.mark.parametrize("kind", [S.SERIAL, S.SKLANSKY, S.KOGGE_STONE, S.BRENT_KUNG, S.BLELLOCH])
def test_schedules_match_oracle(lib, kind):
    for n in list(range(1, 70)) + [127, 399]:
        got, aux = lib.schedule(kind, n)
        assert _norm(got) == _norm(S.schedule(kind, n)), (kind, n)
        assert aux == S.aux_slots(kind, n)


@pytest.mark.parametrize("kind", [S.CHUNKED, S.CHUNKED_ALT])
@pytest.mark.parametrize("gkind", [S.SERIAL, S.SKLANSKY, S.KOGGE_STONE, S.BRENT_KUNG, S.BLELLOCH])
def test_chunked_schedules_match_oracle(lib, kind, gkind):
    for n in [1, 2, 5, 16, 33, 100, 399]:
        for p in [1, 2, 3, 8, 16, 64]:
            got, aux = lib.schedule(kind, n, p, gkind)
            assert _norm(got) == _norm(S.schedule(kind, n, p, gkind)), (kind, gkind, n, p)
            assert aux == S.aux_slots(kind, n, p, gkind)


@pytest.mark.parametrize("k", [1, 2, 3, 9, 30])
def test_han_carlson_schedule_matches_oracle(lib, k):
    for n in list(range(1, 70)) + [127, 128, 399]:
        got, aux = lib.schedule(S.HAN_CARLSON, n, k)
        assert _norm(got) == _norm(S.schedule(S.HAN_CARLSON, n, k)), (k, n)
        assert aux == 0


@pytest.mark.parametrize("k", [0, 1, 2, 3, 9, 30])
def test_ladner_fischer_schedule_matches_oracle(lib, k):
    for n in list(range(1, 70)) + [127, 128, 399]:
        got, aux = lib.schedule(S.LADNER_FISCHER, n, k)
        assert _norm(got) == _norm(S.schedule(S.LADNER_FISCHER, n, k)), (k, n)
        assert aux == 0


def test_invalid_schedule_kind_is_rejected(lib):
    with pytest.raises(lib.RegError):
        lib.schedule(42, 8)


def test_binding_structs_match_the_header(lib, tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets
    that a C compiler gives the header's structures."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"reg_params": lib.Params, "reg_op_desc": lib.OpDesc, "reg_schedule_op": lib.ScheduleOp,
               "reg_kernel_stats": lib.KernelStats, "reg_allocator": lib.Allocator}
    cnames = {"lambda_": "lambda"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "reg.h"', 'int main(void) {']
    want = []
    for cname, py in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {cnames.get(fname, fname)}));')
            want.append(getattr(py, fname).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == want
