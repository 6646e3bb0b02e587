"""The C-ABI library builds, loads and exports every entry point include/pbbem.h declares (no GPU needed)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pbbem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pb_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_declared_symbols():
    from paper_1309_4018_b300.build import build
    lib = build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pb_[a-z0-9_]+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing


def test_binding_loads_and_covers_header():
    import paper_1309_4018_b300.pbbem as pbbem
    assert set(_declared()) <= set(pbbem.EXPORTED)


def test_no_device_is_a_clean_error():
    # on a host without a CUDA device, context creation fails with a status, not a crash
    import paper_1309_4018_b300.pbbem as pbbem
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    try:
        pbbem.Context(0)
    except pbbem.PBError as e:
        assert e.code in (pbbem.PB_ECUDA, pbbem.PB_EINVAL)
    else:
        raise AssertionError("context creation without a device must fail")
