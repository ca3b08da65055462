"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function include/mlkd.h declares; host-side validation needs no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^(?:MLKD_API\s+)?[A-Za-z_][\w \*]*?\b(mlkd_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_2004_04071_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("mlkd_run_level", "mlkd_estimate", "mlkd_debug_pairs", "mlkd_context_create",
                 "mlkd_workspace_bytes"):
        assert want in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(built)
    for n in declared_functions():
        getattr(lib, n)


def test_binding_names_match_header(built):
    import paper_2004_04071_gb300 as mk
    assert sorted(mk.EXPORTED) == sorted(n for n in declared_functions() if n in mk.EXPORTED)
    for n in declared_functions():
        assert n in mk.EXPORTED, n


def test_struct_layouts_match_header(built):
    import paper_2004_04071_gb300 as mk
    # mlkd_problem: 4 doubles, 6 int32, 3 doubles, 2 x 32-bit, u64, pointer, 2 int32, pointer
    assert ctypes.sizeof(mk.Problem) == 4 * 8 + 6 * 4 + 3 * 8 + 8 + 8 + 8 + 8 + 8 + 8 + 3 * 8
    assert ctypes.sizeof(mk.LevelStats) == 8 + 6 * 8 + 2 * 8
    # mlkd_batch_config: 9 int32
    assert ctypes.sizeof(mk.BatchConfig) == 9 * 4
    assert mk.lib().mlkd_abi_version() == mk.ABI_VERSION


def test_validation_without_gpu(built):
    import paper_2004_04071_gb300 as mk
    ok = mk.make_problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=1)
    assert mk.workspace_bytes(ok) > 0
    bad = [dict(eps=0.0), dict(eps=-1.0), dict(T=0.0), dict(dt0=0.3), dict(M=1), dict(M=65),
           dict(L=-1), dict(L=16), dict(nbins=-1), dict(nbins=1025), dict(qoi=7),
           dict(qoi=2, nbins=0), dict(init=3), dict(precision=5), dict(nbins=4, lo=1.0, hi=1.0),
           dict(L=15, M=3, precision=1), dict(L=15, M=4), dict(eps=float("nan"))]
    for b in bad:
        kw = dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=1)
        kw.update(b)
        assert mk.workspace_bytes(mk.make_problem(**kw)) == 0, b
    # 5 * 3^15 fine steps: exact step indices in FP64 state, not in FP32 state
    assert mk.workspace_bytes(mk.make_problem(eps=0.5, T=0.5, dt0=0.1, M=3, L=15)) > 0
    # the caps are inclusive: 2^30 fine steps with FP64 state, 2^24 with FP32 state
    for prec, L, ok_at_cap in [(0, 15, True), (3, 15, True), (1, 12, True), (2, 12, True)]:
        at_cap = mk.make_problem(eps=0.5, T=1.0, dt0=1.0, M=4, L=L, precision=prec)
        over = mk.make_problem(eps=0.5, T=2.0, dt0=1.0, M=4, L=L, precision=prec)
        assert mk.workspace_bytes(at_cap) > 0, (prec, L)
        assert mk.workspace_bytes(over) == 0, (prec, L)
    assert mk.workspace_bytes(mk.make_problem(eps=0.5, T=1.0, dt0=1.0, M=4, L=13, precision=2)) == 0


def test_status_strings(built):
    import paper_2004_04071_gb300 as mk
    assert mk.status_string(0) == "ok"
    assert mk.status_string(mk.MLKD_EINVAL) == "invalid argument"


def test_level_set_validation(built):
    import paper_2004_04071_gb300 as mk
    base = dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=6)
    assert mk.workspace_bytes(mk.make_problem(level_set=[2, 4, 6], **base)) > 0
    assert mk.workspace_bytes(mk.make_problem(level_set=[6], **base)) > 0
    for bad in ([2, 4], [4, 2, 6], [2, 2, 6], [-1, 6], [0, 1, 2, 3, 4, 5, 6, 7]):
        assert mk.workspace_bytes(mk.make_problem(level_set=bad, **base)) == 0, bad
    # a gap may coarsen by at most 2^20
    assert mk.workspace_bytes(mk.make_problem(eps=0.1, T=1.0, dt0=0.5, M=4, L=11,
                                              level_set=[0, 11])) == 0
    assert mk.workspace_bytes(mk.make_problem(eps=0.1, T=1.0, dt0=0.5, M=4, L=11,
                                              level_set=[0, 5, 11])) > 0
