"""The CPU oracle pinned to the paper and to mathematics (no GPU).

Every pin of ``_pins.py`` must hold on the default oracle build, and every
planted-mistake build of the oracle must fail at least one quick pin.
"""
import os

import numpy as np
import pytest

import oracle
import _pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def orc():
    return oracle.load()


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(orc, pin):
    assert orc.mutant == 0
    msg = pin(orc)
    assert msg is None, msg


@pytest.mark.parametrize("mutant", sorted(oracle.MUTANTS))
def test_planted_mistake_is_caught(mutant):
    bad = oracle.load(mutant)
    assert bad.mutant == mutant
    failures = [p.__name__ for p in _pins.QUICK_PINS if p(bad) is not None]
    assert failures, f"planted mistake '{oracle.MUTANTS[mutant]}' passed every pin"


def test_argument_errors(orc):
    counts = np.zeros(8, dtype=np.uint64)
    data = np.zeros(4, dtype=np.uint8)
    assert orc.bytes_rc(3, counts, data.ctypes.data, 4) == oracle.EINVAL
    assert orc.bytes_rc(512, counts, data.ctypes.data, 4) == oracle.EINVAL
    assert orc.bytes_rc(8, counts, None, 4) == oracle.EINVAL
    assert orc.bytes_rc(8, counts, None, 0) == oracle.OK  # n == 0 is a no-op


def _read_fixture(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=", 1)
                rows[k.strip()] = v.strip()
    return rows


def _lop3(imm, a, b, c, width):
    """PTX lop3 semantics: output bit = imm[(a_bit << 2) | (b_bit << 1) | c_bit]."""
    out = 0
    for i in range(width):
        idx = (((a >> i) & 1) << 2) | (((b >> i) & 1) << 1) | ((c >> i) & 1)
        out |= ((imm >> idx) & 1) << i
    return out


def test_full_adder_worked_example_and_truth_tables():
    """Section 3.1's worked full-adder example and the ternary-logic immediates.

    The fixture holds the paper's printed values.  The immediates for sum
    (parity) and carry (majority) are recomputed from their truth tables, then
    applied bitwise to the worked example.
    """
    fx = _read_fixture("full_adder_example.txt")
    a, b, c = (int(fx[k], 2) for k in ("a", "b", "c"))
    carry, summ = int(fx["carry"], 2), int(fx["sum"], 2)
    # the arithmetic fact a full adder encodes: a_i + b_i + c_i == 2*C_i + S_i per bit
    for i in range(4):
        bits = ((a >> i) & 1) + ((b >> i) & 1) + ((c >> i) & 1)
        assert bits == 2 * ((carry >> i) & 1) + ((summ >> i) & 1)
    ta, tb, tc = 0xF0, 0xCC, 0xAA
    parity = ta ^ tb ^ tc
    majority = (ta & tb) | (ta & tc) | (tb & tc)
    mux = (ta & tb) | (~ta & 0xFF & tc)
    assert parity == int(fx["lut_parity"], 16)
    assert majority == int(fx["lut_majority"], 16)
    assert mux == int(fx["lut_mux"], 16)
    assert _lop3(parity, a, b, c, 4) == summ
    assert _lop3(majority, a, b, c, 4) == carry
