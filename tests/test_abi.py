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


def _ctypes_layout():
    """{struct: (size, {field: offset})} of the binding's ctypes mirrors."""
    from paper_1711_03789_gb300 import _lib as L
    mirrors = {"mx_mesh_desc": L.MeshDesc, "mx_dd_desc": L.DdDesc, "mx_coarse_desc": L.CoarseDesc,
               "mx_problem_info": L.ProblemInfo, "mx_rhs_stats": L.RhsStats, "mx_timing": L.Timing,
               "mx_request": L.MxRequest, "mx_request_timing": L.RequestTiming, "mx_server_info": L.ServerInfo}
    import ctypes
    return {name: (ctypes.sizeof(cls), {f: getattr(cls, f).offset for f, _ in cls._fields_})
            for name, cls in mirrors.items()}


def test_c_client_compiles_links_and_matches_the_binding():
    """tests/c/abi_check.c includes the header as strict C99 (-pedantic -Werror), links
    against libmxas.so, checks the argument errors that need no GPU, and prints every ABI
    struct's size and field offsets, which must equal the ctypes mirrors field by field."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    import paper_1711_03789_gb300 as mx
    libdir = os.path.dirname(mx.lib_path)
    out_dir = os.path.join(libdir, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "abi_check")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_check.c"), "-L", libdir, "-lmxas",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    sizes, offsets = {}, {}
    for line in r.stdout.splitlines():
        parts = line.split()
        if parts[0] == "size":
            sizes[parts[1]] = int(parts[2])
        elif parts[0] == "offset":
            s, f = parts[1].split(".")
            offsets.setdefault(s, {})[f] = int(parts[2])
    want = _ctypes_layout()
    assert set(sizes) == set(want)
    for name, (size, fields) in want.items():
        assert sizes[name] == size, name
        assert offsets[name] == fields, name


def test_binding_constants_match_the_header():
    """Every integer #define MX_* and enum value of include/mxas.h has a constant of the same
    name and value in the Python binding."""
    import paper_1711_03789_gb300 as mx
    src = open(os.path.join(ROOT, "include", "mxas.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (MX_\w+)\s+\(?(-?\d+)\)?", src, re.M)}
    for body in re.findall(r"typedef enum \{([^}]*)\}", src):
        for name, val in re.findall(r"(MX_\w+)\s*=\s*(-?\d+)", body):
            consts[name] = int(val)
    assert len(consts) >= 24
    for name, val in consts.items():
        assert getattr(mx, name, None) == val, name
