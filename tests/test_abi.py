"""The C ABI library loads and exports what include/top.h declares (CPU only)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "top.h")


@pytest.fixture(scope="module")
def top():
    from paper_2507_10290_gb300 import build
    build.build()
    from paper_2507_10290_gb300 import top as T
    return T


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(top_\w+)\s*\(", src)))


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("top_create", "top_solve", "top_grad", "top_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(top):
    out = subprocess.run(["nm", "-D", "--defined-only", top.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s+(\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = C.CDLL(top.LIB_PATH)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_struct_layouts_match_the_header(top, tmp_path):
    probe = tmp_path / "probe.c"
    fields = {
        "top_config": [f for f, _ in top.top_config._fields_],
        "top_problem": [f for f, _ in top.top_problem._fields_],
        "top_result": [f for f, _ in top.top_result._fields_],
        "top_state": [f for f, _ in top.top_state._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-o", str(exe), str(probe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for s, cls in (("top_config", top.top_config), ("top_problem", top.top_problem),
                   ("top_result", top.top_result), ("top_state", top.top_state)):
        assert int(got[f"{s} size"]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_error_strings_and_constants(top):
    for code in (top.TOP_OK, top.TOP_E_INVAL, top.TOP_E_NOMEM, top.TOP_E_CUDA, top.TOP_E_TIMEOUT,
                 top.TOP_E_NOTSUP, top.TOP_E_STATE, top.TOP_E_NUMERIC, top.TOP_E_LIMIT, top.TOP_E_BOUNDS):
        s = top.top_strerror(code)
        assert s and s != "unknown error code"
    assert top.top_strerror(12345) == "unknown error code"
    assert top.top_last_cuda_error(None) == 0


def test_create_rejects_bad_configs_without_touching_the_gpu(top):
    cfg = top.top_config()
    cfg.max_batch = 0
    cfg.max_segments = 10
    assert top.top_create(cfg)[0] == top.TOP_E_INVAL
    cfg.max_batch = 1
    cfg.precision = 7
    assert top.top_create(cfg)[0] == top.TOP_E_INVAL
    cfg.precision = 0
    cfg.stream_form = 2
    assert top.top_create(cfg)[0] == top.TOP_E_INVAL
    cfg.stream_form = 0
    cfg.reserved[3] = 1
    assert top.top_create(cfg)[0] == top.TOP_E_INVAL


def test_binding_constants_match_the_header(top):
    """Every #define TOP_* number and enumerator of include/top.h has the same
    value in the Python binding."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(TOP_\w+)\s+\(?(-?\d+)\)?", src)}
    for body in re.findall(r"enum\s+\w+\s*\{([^}]*)\}", src):
        for name, val in re.findall(r"(TOP_\w+)\s*=\s*(-?\d+)", body):
            values[name] = int(val)
    assert len(values) > 30
    missing = [n for n in values if not hasattr(top, n)]
    assert not missing, missing
    wrong = {n: (getattr(top, n), v) for n, v in values.items() if getattr(top, n) != v}
    assert not wrong, wrong


def test_product_package_does_not_reach_the_oracle():
    """The CUDA path never imports, includes or loads anything from oracle/."""
    pkg = os.path.join(ROOT, "paper_2507_10290_gb300")
    pat_py = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|from\s+\.\.oracle)", re.M)
    pat_c = re.compile(r"#\s*include\s*[<\"][^>\"]*oracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                text = open(path).read()
                assert not pat_py.search(text), path
                assert "top_oracle" not in text and "liboracle" not in text, path
            elif f.endswith((".cu", ".cuh", ".h", ".cpp")):
                assert not pat_c.search(open(path).read()), path
