"""CPU checks of the C ABI: the library builds and loads, exports every entry
point include/pslbm.h declares, the ctypes mirror of pslbm_params has the C
layout, and parameter validation rejects bad input before touching a device."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pslbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1410_3464_gb300 import build, pslbm
    build.build()
    return pslbm


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pslbm_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pslbm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    loaded = lib.load()
    for n in names:
        assert hasattr(loaded, n)
    assert set(lib.EXPORTS) <= set(names)


def test_params_layout_matches_c(lib, tmp_path):
    fields = [f for f, _ in lib.Params._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){",
            'printf("%zu\\n", sizeof(pslbm_params));']
    for f in fields:
        prog.append(f'printf("%zu\\n", offsetof(pslbm_params, {f}));')
    prog.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == C.sizeof(lib.Params)
    for f, off in zip(fields, vals[1:]):
        assert getattr(lib.Params, f).offset == off, f


def _create(lib, **over):
    from paper_1410_3464_gb300 import inputs
    sc = inputs.bubble_grain(nx=16, ny=8, grain=(8, 4, 2), bubble=(3, 4, 1))
    p = dict(sc["params"])
    p.update(over)
    return lib.Simulation(sc["mask"], p, sc["rho1"], sc["rho2"], sc["conc"])


@pytest.mark.parametrize("bad", [
    dict(tau=(0.5, 1.0)),
    dict(tau_g=(0.4, 0.8, 1, 1)),
    dict(J0=(1.0, 0.3, 0, 0)),
    dict(n_species=5),
    dict(idx_B=3),
    dict(idx_A=1, idx_B=1),
    dict(k2=0.34),            # kappa = k2 / (2 J_w) >= 1 for J0 = 1/3
    dict(V_split=1.0),
    dict(nx=0),
    dict(precision=7),
])
def test_create_rejects_bad_parameters(lib, bad):
    import numpy as np
    from paper_1410_3464_gb300 import inputs
    sc = inputs.bubble_grain(nx=16, ny=8, grain=(8, 4, 2), bubble=(3, 4, 1))
    p = dict(sc["params"])
    p.update(bad)
    prm = lib.params_from_dict(p)
    buf = np.zeros(16 * 8 * 8)
    h = C.c_void_p()
    ptr = buf.ctypes.data_as(C.c_void_p)
    st = lib.load().pslbm_create(ptr, ptr, ptr, None, None, C.byref(prm), C.byref(h))
    assert st == -1
    assert h.value is None
    assert lib.load().pslbm_last_error(None)


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present")
    with pytest.raises(lib.PslbmError) as e:
        _create(lib)
    assert e.value.status == -8
