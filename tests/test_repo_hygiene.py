"""Repository rules that a test can check on the CPU.

- profiles/ holds text summaries only, and every ncu command in them leaves the
  GPU clocks alone (`--clock-control none`) and runs committed files only.
- The product package never imports the oracle: the FP64 oracle is test
  infrastructure, and the CUDA path has no CPU fallback: without its library,
  or without a CUDA device, the binding raises instead of computing anything.
"""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")
PACKAGE = os.path.join(ROOT, "paper_2408_02367_gb300")


def test_profiles_are_text_summaries():
    for f in os.listdir(PROFILES):
        assert f.endswith((".md", ".txt")), f
        assert os.path.getsize(os.path.join(PROFILES, f)) < 64 * 1024, f


def test_profile_ncu_commands_leave_clocks_alone_and_run_committed_files():
    n = 0
    for f in sorted(os.listdir(PROFILES)):
        for line in open(os.path.join(PROFILES, f)):
            cmd = line.strip()
            if not re.match(r"^ncu\s+-", cmd) or cmd.startswith("ncu -i"):
                continue
            n += 1
            assert "--clock-control none" in cmd, (f, cmd)
            assert "_work/" not in cmd, (f, cmd)
    assert n > 0


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PACKAGE):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                else:
                    continue
                assert not any(nm == "oracle" or nm.startswith("oracle.") for nm in names), (f, names)


def test_binding_fails_loudly_without_its_library_or_a_device(monkeypatch, tmp_path):
    torch = pytest.importorskip("torch")
    from paper_2408_02367_gb300 import op
    monkeypatch.setattr(op, "_LIB", None)
    monkeypatch.setattr(op, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        op.lib()
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            op.SubspaceNufft(torch.zeros((4, 3)), [0, 4], (8, 8, 8), 4, 2.0, torch.zeros((1, 1), dtype=torch.complex64),
                             torch.zeros((1, 8, 8, 8), dtype=torch.complex64))
