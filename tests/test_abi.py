"""The C ABI library builds for sm_103a, loads, and exports every function
include/fast.h declares; the binding covers them.  No GPU calls."""
import ctypes
import os
import re

import paper_2102_10768_gb300 as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fast.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fast_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_pipeline():
    names = declared_functions()
    for f in ("fast_load_graph", "fast_build_cst", "fast_partition", "fast_match"):
        assert f in names


def test_library_exports_every_declared_symbol():
    F.build()
    lib = ctypes.CDLL(F.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(F.exported_symbols()) == declared_functions()


def test_config_default_without_gpu():
    c = F.default_config()
    assert c.delta_w == 1 << 20 and c.warps_per_block == 8 and c.max_chunks == 1 << 16 and c.limit == 0
    assert c.queue_cells == 0 and c.order_rule == 0 and c.filter_rule == 0 and c.build_rule == 0
    assert c.refine_rule == 0 and c.matcher_rule == 0 and c.validators == 0
    # fast_config_default zeroes exactly sizeof(fast_config) bytes, so a
    # sentinel-filled buffer shows the C size; it must be the binding's
    buf = (ctypes.c_ubyte * 256)(*([0xAB] * 256))
    F.lib().fast_config_default(ctypes.byref(buf))
    c_size = next(i for i in range(256) if buf[i] == 0xAB)
    assert c_size == ctypes.sizeof(F.Config) == 96
    assert F.lib().fast_last_error() == b""


def test_config_rejects_unknown_fields():
    import pytest
    with pytest.raises(TypeError):
        F.default_config(fiter_rule=1)
    c = F.default_config(filter_rule=1, build_rule=1)
    assert c.build_rule == 1
    with pytest.raises(AttributeError):
        c.bulid_rule = 1


def test_injected_allocation_failure_fires_once():
    """fast_inject_alloc_failure(0): the next device allocation fails with
    FAST_ERR_OOM and says it was injected; the injector is then off, so the
    next call reaches a real allocation (which, on a machine without a GPU,
    fails for that reason instead)."""
    import numpy as np
    import pytest
    e = np.array([[0, 1], [1, 2]], np.int32)
    lab = np.zeros(4, np.int32)
    assert F.inject_alloc_failure(0) == -1
    try:
        with pytest.raises(F.FastError, match="injected"):
            F.Graph(4, e, lab)
    finally:
        assert F.inject_alloc_failure(-1) == -1           # it fired
    assert F.inject_alloc_failure(7) == -1 and F.inject_alloc_failure(-1) == 7
    try:
        F.Graph(4, e, lab)
    except F.FastError as err:
        assert "injected" not in str(err)


def test_every_kernel_launch_is_counted():
    """fast_kernel_launches (the bench's gpu_launches) counts every launch the
    library makes: each `<<<` in its sources is followed by note_launch()
    within a few lines."""
    import glob
    missing = []
    for path in sorted(glob.glob(os.path.join(ROOT, "paper_2102_10768_gb300", "csrc", "*.cu*"))):
        lines = open(path).read().split("\n")
        for i, ln in enumerate(lines):
            if "<<<" not in ln or ln.lstrip().startswith("//"):
                continue
            window = "\n".join(lines[i:i + 6])
            if "note_launch(" not in window:
                missing.append(f"{os.path.basename(path)}:{i + 1}")
    assert not missing, missing


def test_product_never_imports_the_oracle():
    """The library's package never imports oracle/; bench.py imports it only
    inside its CPU baseline and reference arm."""
    import ast
    import glob

    def oracle_imports(tree):
        for node in ast.walk(tree):
            if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                yield node
            if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                yield node

    for path in glob.glob(os.path.join(ROOT, "paper_2102_10768_gb300", "**", "*.py"), recursive=True):
        assert not list(oracle_imports(ast.parse(open(path).read()))), path
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef) and fn.name in ("cpu_baseline", "run_reference", "oracle_sample"):
            allowed |= {id(n) for n in oracle_imports(fn)}
    assert all(id(n) in allowed for n in oracle_imports(tree))


def test_oracle_and_library_share_no_code():
    """No library source includes an oracle file and no oracle source includes
    a library file (they meet only through synth/'s inputs and the tests)."""
    import glob
    import re
    inc = re.compile(r'#\s*include\s*"([^"]+)"')
    for path in glob.glob(os.path.join(ROOT, "paper_2102_10768_gb300", "csrc", "*")):
        for name in inc.findall(open(path).read()):
            assert "oracle" not in name, (path, name)
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        for name in inc.findall(open(path).read()):
            assert "csrc" not in name and "fast.h" not in name and "internal" not in name, (path, name)
