"""The C ABI library builds, loads without a GPU and exports every entry point include/sk.h
declares (no compute calls: this runs on CPU-only machines)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "sk.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"SK_API\s+[\w\s\*]+?\b(sk_\w+)\s*\(", src)))


def test_header_declares_expected_set():
    from paper_2606_20195_gb300 import sk
    assert _declared() == sorted(sk.EXPORTS)


def test_library_exports_every_declared_symbol():
    from paper_2606_20195_gb300 import _build, sk
    lib = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(sk_\w+)", out))
    for name in _declared():
        assert name in exported, name
    L = sk.load(lib)
    for name in _declared():
        assert hasattr(L, name)
    assert L.sk_version() >= 10000


def test_plan_validation_runs_without_gpu():
    # sk_plan_create is host-only: argument checks work on a CPU-only machine.
    from paper_2606_20195_gb300 import sk
    sk.load()
    import pytest
    with pytest.raises(sk.SkError) as e:
        sk.sk_plan_create(10, 100, 4, 0, 0)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    h = sk.sk_plan_create(4096, 1 << 22, 8, sk.SK_FP16_RN, 7)
    sk.sk_plan_set(h, sk.SK_PARAM_CHUNK_ROWS, 4096)
    assert sk.sk_plan_get(h, sk.SK_PARAM_CHUNK_ROWS) == 4096
    assert sk.sk_plan_get(h, sk.SK_PARAM_SOLVE_GROUP_ROWS) == 0
    sk.sk_plan_set(h, sk.SK_PARAM_SOLVE_GROUP_ROWS, 96)
    assert sk.sk_plan_get(h, sk.SK_PARAM_SOLVE_GROUP_ROWS) == 96
    with pytest.raises(sk.SkError) as e:
        sk.sk_plan_set(h, sk.SK_PARAM_SOLVE_GROUP_ROWS, -1)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    sk.sk_destroy(h)


def test_binding_constants_match_header():
    # every named constant of include/sk.h (status codes, rules, parameter keys, modes, kernels,
    # element types) has the same value in the Python binding
    from paper_2606_20195_gb300 import sk
    with open(os.path.join(ROOT, "include", "sk.h")) as f:
        src = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    consts = dict((name, int(val)) for name, val in re.findall(r"\b(SK_[A-Z0-9_]+)\s*=\s*(\d+)", src))
    assert len(consts) >= 30
    missing = [c for c in consts if not hasattr(sk, c)]
    assert not missing, missing
    wrong = {c: (v, getattr(sk, c)) for c, v in consts.items() if getattr(sk, c) != v}
    assert not wrong, wrong
