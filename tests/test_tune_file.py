"""The tune-file parser, checked on the host (no GPU): the shipped table,
per-width entries, and the line numbers of malformed lines."""
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHIPPED = os.path.join(ROOT, "paper_2412_16370_gb300", "pospopcnt_tune.txt")


@pytest.fixture(scope="module")
def pp():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2412_16370_gb300 import build, binding
    build.build()
    return binding


def _check(pp, tmp_path, text):
    f = tmp_path / "t.txt"
    f.write_text(text)
    return pp.pospopcnt_tune_check(str(f))


def test_shipped_table_parses(pp):
    assert pp.pospopcnt_tune_check(SHIPPED) == 0


def test_empty_and_comment_only_files_parse(pp, tmp_path):
    assert _check(pp, tmp_path, "") == 0
    assert _check(pp, tmp_path, "# nothing here\n\n   \n") == 0


def test_per_width_and_every_width_entries(pp, tmp_path):
    lines = ["stream 0 256 2 16 1 1 2"]                 # every width
    for w in (8, 16, 32, 64):
        lines.append(f"stream {w} 1 128 4 32 0 3 1")    # one width group
        lines.append(f"batch {w} 512 1 16 1 1 127 1")
    lines += ["batch 256 2 16 0 2 63 4", "pdl 0", "staged 0", "short 1", "split 1024",
              "roofline 256 1 18", "wait 0", "wait 2147483648",
              "serve 0 8 127 64 1024", "serve 3 0 127 1 1", "serve_light 0",
              "serve_light 536870912", "batch_rows 1 8 127 511", "batch_rows 16 2 16 255 2047",
              "serve_strided 1", "serve_strided 0", "serve_order 1", "multi 8 0",
              "serve_promote 0", "serve_promote 250", "serve_shape 512 1 16 0",
              "serve_mode 1", "serve_mode 2", "serve_mode 0", "serve_srf 268435456 4 255", "serve_srf 512 1 1",
              "serve_srf 134217728 4 0", "serve_srf_class 31 127 0 0", "serve_srf_age 150", "serve_srf_age 0", "serve_mode 3", "serve_resident 2000 200000", "serve_resident 1 1",
              "serve_shape 256 2 32 1",
              "multi 1048576 1",
              "stream 4 512 1 16 0 3 1   # trailing comment"]
    assert _check(pp, tmp_path, "\n".join(lines) + "\n") == 0
    assert _check(pp, tmp_path, "\r\n".join(lines) + "\r\n") == 0   # CRLF line ends


@pytest.mark.parametrize("bad", [
    "stream 24 2 512 1 16 1 1 8",        # 24 is not a width group
    "stream 128 2 512 1 16 1 1 8",       # groups are named by 8, 16, 32, 64
    "stream 5 512 1 16 1 1 8",           # size class out of range
    "stream 8 2 512 1 16 1 1",           # seven fields: class 8 out of range
    "stream 0 512 1 16 1 1",             # too few fields
    "stream 8 2 512 1 16 1 1 8 9",       # too many
    "stream 0 500 1 16 1 1 8",           # no such block shape
    "stream 0 512 1 24 1 1 8",           # no such flush depth
    "stream 0 512 1 16 1 0 8",           # ctas per SM below 1
    "stream 0 512 1 16 1 1 0",           # rows per warp below 1
    "stream 0 512 1 16 1 1 x",           # not an integer
    "stream 0 512 1 16 1 -1 8",          # negative
    "batch 512 1 16 1 1 0 1",            # item rows below 1
    "batch 512 1 16 1 1 2097152 1",      # item rows above 2^20
    "batch 512 1 16 1 1 127 65",         # grab above 64
    "batch 64 512 1 16 1 1 127 1 1",     # too many fields
    "pdl 2", "pdl 1 1", "pdl", "pdl -1", "short 2", "short 1 x", "split 0", "split 67108865",
    "split 4 x", "staged 99", "staged", "roofline 300 1 4", "roofline 256 1",
    "roofline 256 1 18 5", "roofline 256 1 0", "bogus 1",
    "wait -1", "wait 2147483649", "wait", "wait 5 5", "wait x",
    "serve 4 8 127 8 1024",              # no such serving class
    "serve 0 8 0 8 1024",                # rows below 1
    "serve 0 8 127 0 1024",              # streams below 1
    "serve 0 8 127 65 1024",             # streams above 64
    "serve 0 8 127 8 1025",              # batch cap above 1024
    "serve 0 8 127 8", "serve_light", "serve_light -5",
    "batch_rows 1 8 127", "batch_rows 24 1 8 127 511", "batch_rows 0 8 127 511",
    "batch_rows 1 8 127 2097152", "batch_rows 16 1 8 127 511 9",
    "serve_strided 2", "serve_strided", "serve_strided 1 1",
    "serve_order 2", "serve_order", "multi 7 0", "multi 1048577 0", "multi 4096 2", "multi 4096",
    "serve_promote -1", "serve_promote 10000001", "serve_promote",
    "serve_shape 500 1 16 0", "serve_shape 512 1 16", "serve_shape 512 1 24 0",
    "serve_mode 4", "serve_srf_age -1", "serve_srf_age 10000001", "serve_srf_class 1 2 3", "serve_srf_class 1 2 3 1048577", "serve_srf 511 1 1", "serve_srf 511 1 0", "serve_resident 0 5", "serve_resident 5", "serve_srf 1048576 4 -1", "serve_srf 268435456 0 255", "serve_srf 268435456 4",
])
def test_malformed_line_is_reported_with_its_number(pp, tmp_path, bad):
    text = "# header\nstream 0 256 2 16 1 1 2\n\n" + bad + "\npdl 1\n"
    assert _check(pp, tmp_path, text) == 4


def test_unreadable_file_raises(pp, tmp_path):
    with pytest.raises(pp.PospopError):
        pp.pospopcnt_tune_check(str(tmp_path / "missing.txt"))
