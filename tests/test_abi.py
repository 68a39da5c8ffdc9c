"""The C ABI libraries build, load and export every symbol their headers declare (no GPU)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

HEADERS = {
    "pospopcnt.h": "libpospopcnt.so",
    "pospop_synth.h": "libpospop_synth.so",
}


def _declared(header: str) -> list[str]:
    text = open(os.path.join(INCLUDE, header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(pospop\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libs():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2412_16370_gb300 import build
    return dict(zip(("libpospopcnt.so", "libpospop_synth.so"), build.build()))


@pytest.mark.parametrize("header", sorted(HEADERS))
def test_every_declared_symbol_is_exported(libs, header):
    names = _declared(header)
    assert len(names) >= 4, names
    path = libs[HEADERS[header]]
    lib = ctypes.CDLL(path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    nm = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True)
    if nm.returncode == 0:
        exported = set(re.findall(r"\bT (pospop\w+)", nm.stdout))
        assert set(names) <= exported


def test_header_compiles_as_c(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "t.c"
    src.write_text('#include "pospopcnt.h"\n#include "pospop_synth.h"\nint main(void){return 0;}\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", INCLUDE, "-c", str(src),
                        "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_strerror_without_gpu(libs):
    from paper_2412_16370_gb300 import binding
    assert "invalid" in binding.strerror(binding.POSPOP_EINVAL)
    assert binding.strerror(12345) == "unknown status code"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2412_16370_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.pospopcnt_launch_count()


def test_no_oracle_on_the_product_path():
    """The package never imports, loads or calls the oracle."""
    pkg = os.path.join(ROOT, "paper_2412_16370_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f), errors="replace").read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text and "oracle_pospop" not in text, f
