"""Structural rules checked on the CPU: the product path and the oracle
share no code and do not import each other, the Python status codes match
the C header, the header compiles as C and as C++, and the binding fails
loudly (no fallback) when the library is missing."""
import ast
import os
import re
import subprocess

import pytest

import paper_2602_10080_gb300 as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sssp.h")


def _python_imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
    return names


def _files(sub, exts):
    for dirpath, _, files in os.walk(os.path.join(ROOT, sub)):
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_product_never_imports_or_includes_the_oracle():
    for path in _files("paper_2602_10080_gb300", (".py",)):
        assert "oracle" not in _python_imports(path), path
    for path in _files("paper_2602_10080_gb300", (".cu", ".cuh", ".h", ".cpp")):
        text = open(path).read()
        assert not re.search(r'#include\s+["<][^">]*oracle', text), path
        assert "sssp_oracle" not in text, path


def test_oracle_never_imports_the_product():
    for path in _files("oracle", (".py",)):
        assert "paper_2602_10080_gb300" not in _python_imports(path), path
    for path in _files("oracle", (".c", ".h")):
        text = open(path).read()
        assert "mlmq" not in text and "sssp.h" not in text, path


def test_status_codes_match_header():
    text = open(HEADER).read()
    codes = dict((m.group(1), int(m.group(2))) for m in re.finditer(r"#define (SSSP_E_\w+)\s+(-?\d+)", text))
    codes["SSSP_OK"] = int(re.search(r"#define SSSP_OK\s+(\d+)", text).group(1))
    for name, value in codes.items():
        assert getattr(S, name) == value, name
    S.lib()
    unknown = S.strerror(-12345)
    for name, value in codes.items():
        msg = S.strerror(value)
        assert msg and msg != unknown, (name, msg)


@pytest.mark.parametrize("lang,compiler", [("c", "gcc"), ("c++", "g++")])
def test_header_compiles(tmp_path, lang, compiler):
    src = tmp_path / ("use." + ("c" if lang == "c" else "cpp"))
    src.write_text(f'#include "{HEADER}"\nint main(void) {{ sssp_config c; return sssp_config_default(&c) == 0 ? 0 : 1; }}\n')
    r = subprocess.run([compiler, "-x", lang, "-Wall", "-Werror", "-c", str(src), "-o", str(tmp_path / "use.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(S, "_lib", None)
    monkeypatch.setattr(S, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        S.lib()
