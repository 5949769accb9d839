"""Without the compiled library the binding refuses to load: there is no CPU
fallback for any step of the method."""
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_binding_raises_without_the_library(tmp_path):
    pkg = tmp_path / "pkg_without_lib"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_1403_7394_gb300", "hap.py"), pkg / "hap.py")
    (pkg / "__init__.py").write_text("")
    code = "import pkg_without_lib.hap"
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=tmp_path, timeout=300)
    assert out.returncode != 0
    assert "ImportError" in out.stderr and "libhap.so is missing" in out.stderr
