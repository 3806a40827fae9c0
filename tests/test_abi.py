"""Host-side checks of the C ABI (no GPU needed): the shared library loads and exports
every function declared in include/spai_gb300.h, and the Python binding wraps exactly
those names.  Also checks that the product package never imports the oracle."""

import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spai_gb300.h")
PKG = os.path.join(ROOT, "paper_1809_06574_gb300")


def declared_functions():
    text = open(HEADER).read()
    names = re.findall(r"^SPAI_API\s+[\w\s\*]+?\b(\w+)\s*\(", text, flags=re.M)
    assert names, "no declarations found"
    return names


@pytest.fixture(scope="module")
def library():
    import ctypes

    from paper_1809_06574_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ("spai_build", "spai_update", "block_solve", "spai_ctx_create",
                     "spai_assemble", "spai_pc_export", "spai_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(library):
    missing = [n for n in declared_functions() if not hasattr(library, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    import paper_1809_06574_gb300 as sg
    for n in declared_functions():
        assert callable(getattr(sg, n, None)), n


def test_product_never_imports_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    assert all(not a.name.startswith("oracle") for a in node.names), f
                elif isinstance(node, ast.ImportFrom):
                    assert not (node.module or "").startswith("oracle"), f


def test_binding_fails_loudly_without_library(monkeypatch):
    import paper_1809_06574_gb300 as sg
    monkeypatch.setattr(sg, "_lib", None)
    monkeypatch.setattr(sg, "LIB_PATH", "/nonexistent/libspai_gb300.so")
    with pytest.raises(RuntimeError):
        sg.lib()


def test_shifted_coefficients_match_oracle(library):
    """The library forms the coefficients of A(p, s) itself (host code, no GPU needed): they
    equal the oracle's Rayleigh-damped coefficients (D = 0.05 M + 0.01 K(p)) bit for bit, and
    the binding does no arithmetic of its own."""
    import oracle
    import paper_1809_06574_gb300 as sg
    import synth
    w = synth.plain_2d_32()
    for p, s in ((0.1, 1.0), (0.7, 0.5), (1.0, 2.0), (0.123456789, 1.7), (0.0, 0.0), (2.0, 1e-3)):
        assert sg.spai_shifted_coefficients(p, s, w.alpha, w.beta) == oracle.coefficients(p, s), (p, s)
    # several parameters: K(p) = K_0 + p_1 K_1 + p_2 K_2
    c = sg.spai_shifted_coefficients([0.5, 0.25], 2.0, 0.1, 0.2)
    assert c == [2.0 * 2.0 + 0.1 * 2.0, 1.0 + 0.2 * 2.0, (1.0 + 0.2 * 2.0) * 0.5, (1.0 + 0.2 * 2.0) * 0.25]
    with pytest.raises(sg.SpaiError):
        sg.spai_shifted_coefficients(float("nan"), 1.0, 0.05, 0.01)
    assert not hasattr(sg, "affine_coefficients")


def test_column_variant_table_is_host_logic(library):
    """The column-kernel variant table needs no GPU: the register-tiled codes (>= 64) are
    offered exactly for the small tiles they hold (rows <= 32, |J| <= 13), the default is
    a shared-memory team, and pinning round-trips (code 0 clears; a code that does not
    fit the shape is refused)."""
    import paper_1809_06574_gb300 as sg
    for low in (0, 1):
        small = sg.spai_column_variants(low, 25, 13)
        assert small and small[0] < 64 and any(c >= 64 for c in small)
        wide = sg.spai_column_variants(low, 125, 27)
        assert wide and all(c < 64 for c in wide)
        assert sg.spai_column_variants(low, 3000, 3000) == []
    assert sg.spai_column_variant_get(1, 25, 13) == 0
    code = max(sg.spai_column_variants(1, 25, 13))
    sg.spai_column_variant_set(1, 25, 13, code)
    assert sg.spai_column_variant_get(1, 32, 13) == code  # the same row class (25 -> 32)
    assert sg.spai_column_variant_get(1, 33, 13) == 0
    with pytest.raises(sg.SpaiError):
        sg.spai_column_variant_set(1, 125, 27, code)  # a register tile cannot hold 125 x 27
    sg.spai_column_variant_set(1, 25, 13, 0)
    assert sg.spai_column_variant_get(1, 25, 13) == 0


def test_adaptive_defaults_agree():
    """The adaptive SPAI's documented defaults (tolerance 1e-4, 5 steps of 5 columns, 128
    rows) are the same in the header, the binding and the oracle."""
    import inspect

    import oracle
    import paper_1809_06574_gb300 as sg
    text = open(HEADER).read()
    assert "opts NULL: eps 1e-4, max_steps 5, max_new 5,\n * max_rows 128" in text
    b = inspect.signature(sg.spai_build_adaptive).parameters
    o = inspect.signature(oracle.spai_adaptive_pattern).parameters
    for name, val in (("eps", 1e-4), ("max_steps", 5), ("max_new", 5), ("max_rows", 128)):
        assert b[name].default == val and o[name].default == val, name


def test_device_code_never_traps_or_batches_copies():
    """Device-side failures are reported through the error word and bounded waits, never
    by trapping; copies are issued one by one (no batched-copy runtime calls)."""
    csrc = os.path.join(PKG, "csrc")
    for name in os.listdir(csrc):
        text = open(os.path.join(csrc, name)).read()
        assert "__trap" not in text and "trap;" not in text, name
        assert "assert(" not in text.replace("static_assert(", ""), name
        assert "Batch" + "Async" not in text, name
