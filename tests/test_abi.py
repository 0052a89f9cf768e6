"""The C-ABI library loads and exports every entry point include/bps.h declares,
and the ctypes binding matches every prototype and struct of the header
(no compute: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "bps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bps_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1306_1821_gb300 import bps
    from paper_1306_1821_gb300 import build as b
    if not os.path.exists(bps.LIB_PATH):
        b.build()
    return bps.load()


def test_header_declares_the_path():
    names = declared()
    for n in ["bps_create", "bps_set_data", "bps_set_state", "bps_get_state", "bps_hmc_step",
              "bps_sample_power", "bps_sample_bias_norm", "bps_jump", "bps_gibbs_iterate",
              "bps_last_error", "bps_destroy"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1306_1821_gb300 import bps
    for n in declared():
        assert hasattr(lib, n), n
        assert n in bps.declared_symbols(), f"binding lacks {n}"


def test_version_without_gpu(lib):
    assert lib.bps_version().decode().startswith("bps")


def test_staged_upload_takes_the_callers_arrays_unconverted():
    # the library copies the caller's memory after the call returns, so the
    # binding must not hand it a temporary conversion
    import numpy as np

    from paper_1306_1821_gb300 import bps
    ok_c, ok_r = np.zeros(8, np.uint16), np.zeros(8, np.float32)
    for c, r in ((np.zeros(8, np.int32), ok_r), (ok_c, np.zeros(8, np.float64)), (ok_c, np.zeros(16, np.float32)[::2])):
        with pytest.raises(TypeError):
            bps.bps_stage_data_host_u16(None, c, r)


def test_z_pass_bytes_counts_the_line_supports():
    # bench.py's algorithmic bytes of the force z pass, against a direct count:
    # W read on lines that meet the survey, W written on all lines, a and c over
    # each line's support [first & ~3, (last + 4) & ~3)
    import sys

    import numpy as np
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
    import bench
    N = 8
    rng = np.random.default_rng(1)
    R = np.zeros((2, N, N, N), np.float32)
    R[0, 1, 2, 3] = 1.0                 # line (1, 2): voxels 3..3 -> [0, 4)
    R[1, 1, 2, 6] = 0.5                 # same line, other subsample: ... 6 -> [0, 8)
    R[0, 4, 4, 1:3] = 2.0               # line (4, 4): voxels 1..2 -> [0, 4)
    R[1, 7, 0, 4:6] = rng.random(2) + 0.1   # line (7, 0): voxels 4..5 -> [4, 8)
    total, info = bench.z_pass_bytes(R, N)
    row = (N // 2 + 1) * 8
    lines, span = 3, 8 + 4 + 4
    assert total == row * (lines + N * N) + 2 * 4 * span
    assert info["lines_with_support"] == lines / (N * N)
    assert info["support_voxels"] == span / N ** 3
    # a survey that covers every voxel costs the dense pass
    dense = bench.z_pass_bytes(np.ones((1, N, N, N), np.float32), N)[0]
    assert dense == info["dense_bytes"] == 2 * row * N * N + 2 * 4 * N ** 3


def test_last_error_is_per_thread(lib):
    # context-free calls that fail on their arguments (no GPU work): each thread
    # reads its own failure, not the one another thread made in between
    import ctypes
    import threading

    from paper_1306_1821_gb300 import bps
    gate = threading.Barrier(2)
    seen = {}

    def bias_law_fails():
        assert lib.bps_bias_law(-1, None, 1.2, -20.83, 0.895, 0.105, -0.04, None) == bps.BPS_EINVAL
        gate.wait()          # the other thread fails now
        gate.wait()
        seen["a"] = lib.bps_last_error(None).decode()

    def tables_fail():
        gate.wait()
        sp = bps.bps_schechter(-20.44, -1.05, 14.5, 17.77, 0.24)
        assert lib.bps_schechter_tables(ctypes.byref(sp), 0, None, 1.0, 2, None, None) == bps.BPS_EINVAL
        gate.wait()
        seen["b"] = lib.bps_last_error(None).decode()

    ts = [threading.Thread(target=bias_law_fails), threading.Thread(target=tables_fail)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(30)
    assert seen["a"].startswith("bps_bias_law"), seen
    assert seen["b"].startswith("bps_schechter_tables"), seen


def _header_without_comments():
    txt = open(os.path.join(ROOT, "include", "bps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    return "\n".join(ln for ln in txt.splitlines() if not ln.lstrip().startswith("#"))


_SCALAR = {"int": "c_int", "double": "c_double", "float": "c_float", "uint64_t": "c_uint64", "size_t": "c_size_t",
           "bps_status": "c_int"}


def _scalar(t):
    """(bytes, 'f' | 'i' | 'u') of a ctypes scalar type: c_uint64 and c_size_t
    are one class on LP64 systems, so types are compared by width and kind."""
    import ctypes
    if t in (ctypes.c_float, ctypes.c_double):
        return ctypes.sizeof(t), "f"
    return ctypes.sizeof(t), "u" if t(-1).value > 0 else "i"


def _kind_of_c(decl):
    """'pointer', 'char_p' or the (width, kind) of a C parameter / return type."""
    import ctypes
    decl = decl.replace("const ", "").strip()
    if "*" in decl:
        return "char_p" if re.fullmatch(r"char\s*\*", decl) else "pointer"
    return _scalar(getattr(ctypes, _SCALAR[decl.split()[0]]))


def _kind_of_ctypes(t):
    import ctypes
    if t is None:
        return "void"
    if t is ctypes.c_char_p:
        return "char_p"
    if t is ctypes.c_void_p or issubclass(t, ctypes._Pointer):
        return "pointer"
    return _scalar(t)


def test_binding_signatures_match_the_header():
    # every prototype's arity, argument kinds (pointer or the exact scalar width)
    # and return type against the binding's ctypes declarations
    from paper_1306_1821_gb300 import bps
    txt = _header_without_comments()
    protos = re.findall(r"([A-Za-z_][\w\s\*]*?)\b(bps_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", txt)
    assert len(protos) == len(declared())
    for ret, name, params in protos:
        argtypes, restype = bps._SIGS[name]
        params = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        want = [_kind_of_c(re.sub(r"\b\w+$", "", p)) for p in params]
        got = [_kind_of_ctypes(t) for t in argtypes]
        assert got == want, (name, got, want)
        r = ret.strip()
        assert _kind_of_ctypes(restype) == ("void" if r == "void" else _kind_of_c(r)), name


def test_binding_structs_match_the_header():
    import ctypes

    from paper_1306_1821_gb300 import bps
    txt = _header_without_comments()
    structs = dict((name, body) for body, name in re.findall(r"typedef struct\s*\{([^}]*)\}\s*(\w+)\s*;", txt))
    assert set(structs) == {"bps_config", "bps_move_info", "bps_schechter"}
    for name, body in structs.items():
        fields = [f.strip().rsplit(None, 1) for f in body.split(";") if f.strip()]
        cls = getattr(bps, name)
        assert [n for _, n in fields] == [n for n, _ in cls._fields_], name
        assert [_kind_of_c(t) for t, _ in fields] == [_kind_of_ctypes(t) for _, t in cls._fields_], name
    # the C layout of the configuration: natural alignment, 64 bytes
    assert ctypes.sizeof(bps.bps_config) == 64
    assert bps.bps_config.seed.offset == 56
