"""The C-ABI library loads and exports every entry point declared in include/mxas.h
(no compute: runs without a GPU), and host-side argument checks fail cleanly."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mxas.h")).read()
    return sorted(set(re.findall(r"^MX_API\s+[\w\s\*]+?\b(mx_\w+)\(", src, flags=re.M)))


def test_header_parses():
    names = _declared()
    assert "mx_build_problem" in names and "mx_solve" in names and len(names) >= 20


def test_library_exports_every_symbol():
    import paper_1711_03789_gb300 as mx
    for name in _declared():
        assert hasattr(mx.lib, name), name
        assert hasattr(mx, name), f"binding misses {name}"
    assert mx.mx_version().startswith("mxas")


def test_invalid_descriptors_rejected_without_gpu_work():
    import paper_1711_03789_gb300 as mx
    for args in [(0, 1.0, 0.0, 1.0), (4, -1.0, 0.0, 1.0), (4, 1.0, 0.0, 0.0)]:
        with pytest.raises(mx.MxError) as e:
            mx.mx_build_problem(*args)
        assert e.value.code == mx.MX_EINVAL
    with pytest.raises(mx.MxError) as e:
        mx.mx_build_problem(10, 1.0, 0.0, 1.0, 5, 1, coarse_cells=3)  # 3 does not divide 10
    assert e.value.code == mx.MX_EINVAL
