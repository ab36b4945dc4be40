"""The product path's boundary, checked on the CPU: the package never reaches
the oracle (no import, no load of its library), and the binding refuses to
run when the CUDA library is absent instead of falling back to anything."""
import ast
import pathlib

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_2606_04292_gb300"


def _package_sources():
    files = sorted(p for p in PKG.rglob("*.py") if "__pycache__" not in p.parts)
    assert files, "package sources not found"
    return files


def test_package_never_imports_the_oracle():
    for path in _package_sources():
        tree = ast.parse(path.read_text(), filename=str(path))
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""] + [a.name for a in node.names]
            else:
                continue
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (path, names)


def test_package_never_loads_the_oracle_library():
    for path in _package_sources():
        text = path.read_text()
        assert "liborc" not in text and "richards_oracle" not in text, path


def test_cuda_sources_share_nothing_with_the_oracle():
    """No CUDA or C-ABI source includes an oracle header (the two sides share
    no code: tables, helpers or constants)."""
    sources = list((PKG / "csrc").glob("*.cu")) + list((PKG / "csrc").glob("*.cuh")) + \
        list((PKG / "csrc").glob("*.h")) + list((ROOT / "include").glob("*.h"))
    assert sources
    for path in sources:
        for line in path.read_text().splitlines():
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line and "orc" not in line.split("#include", 1)[1], (path, line)


def test_binding_raises_without_the_cuda_library(monkeypatch, tmp_path):
    from paper_2606_04292_gb300 import build as B
    from paper_2606_04292_gb300 import richards as R
    monkeypatch.setattr(B, "LIB", str(tmp_path / "absent" / "librichards_gb300.so"))
    monkeypatch.setattr(R, "_lib", None)
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        R.lib(build_if_missing=False)
