"""Host check of the counting kernels' carry-save-adder networks.

The full-adder wiring of CSA_15 and CSA_16+4 (Section 4.2) is read from the
kernels' own source (the `fa(sum, carry, a, b, c)` lines of `csa15` and
`csa16` in pospop_device.cuh) and simulated bitwise on Python integers, one
bit per input combination, over every combination of the input bits:

* CSA_15: 15 weight-1 inputs (2^15 combinations) must give
  8*a8 + 4*a4 + 2*a2 + a1 = the number of set inputs, with 11 full adders
  and a critical path of 5 (Section 4.2's figures);
* CSA_16+4: the weight-1, -2, -4, -8 planes plus 16 weight-1 inputs
  (2^20 combinations) must give 16*a16 + 8*a8' + 4*a4' + 2*a2' + a1' =
  a1 + 2*a2 + 4*a4 + 8*a8 + the number of set inputs, with 15 full adders.

A full adder is simulated with the lop3 truth tables the kernels use
(0x96 for the sum, 0xe8 for the carry, Eq. 3), so a wrong immediate, a
miswired adder or a dropped input fails here without a GPU.
"""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2412_16370_gb300", "csrc", "pospop_device.cuh")


def _source():
    with open(SRC) as f:
        return f.read()


def _body(src, name):
    m = re.search(r"__device__ __forceinline__ \w+ " + name + r"\(Planes &p, const V4 \*v\) \{", src)
    assert m, name
    depth, i = 1, m.end()
    while depth:
        depth += {"{": 1, "}": -1}.get(src[i], 0)
        i += 1
    return src[m.end():i - 1]


def _adders(body):
    return re.findall(r"\bfa\(\s*([\w.\[\]]+)\s*,\s*([\w.\[\]]+)\s*,\s*([\w.\[\]]+)\s*,"
                      r"\s*([\w.\[\]]+)\s*,\s*([\w.\[\]]+)\s*\)", body)


def _lut(src, name):
    m = re.search(name + r"\(uint32_t a, uint32_t b, uint32_t c\) \{.*?lop3\.b32[^;]*?(0x[0-9a-fA-F]+);",
                  src, re.S)
    assert m, name
    return int(m.group(1), 16)


def _lop3(imm, a, b, c, mask):
    """Bitwise ternary function with truth table imm (lop3 convention:
    index = 4*a + 2*b + c)."""
    out = 0
    for idx in range(8):
        if (imm >> idx) & 1:
            ta = a if idx & 4 else ~a
            tb = b if idx & 2 else ~b
            tc = c if idx & 1 else ~c
            out |= ta & tb & tc
    return out & mask


def _simulate(adders, env, mask, sum_lut, carry_lut):
    depth = {k: 0 for k in env}
    for s, k, a, b, c in adders:
        va, vb, vc = env[a], env[b], env[c]
        d = 1 + max(depth[a], depth[b], depth[c])
        env[s] = _lop3(sum_lut, va, vb, vc, mask)
        env[k] = _lop3(carry_lut, va, vb, vc, mask)
        depth[s] = depth[k] = d
    return env, depth


def _input_patterns(n):
    """n bit-parallel variables covering all 2^n combinations: bit j of
    variable i is bit i of j."""
    size = 1 << n
    out = []
    for i in range(n):
        half = 1 << i
        pat, length = ((1 << half) - 1) << half, 2 * half   # 2^i zeros, then 2^i ones
        while length < size:
            pat |= pat << length
            length *= 2
        out.append(pat)
    return out


def _popcounts(vars_, size):
    """Per combination, the number of set variables, as bit planes of
    weights 1, 2, 4, ... (a bitwise ripple counter over the variables)."""
    mask = (1 << size) - 1
    count = [0] * 6
    for v in vars_:
        carry = v
        for j in range(len(count)):
            count[j], carry = (count[j] ^ carry) & mask, count[j] & carry
            if not carry:
                break
    return count


@pytest.fixture(scope="module")
def src():
    return _source()


def test_lop3_immediates_are_parity_and_majority(src):
    s, k = _lut(src, "lop3_parity"), _lut(src, "lop3_majority")
    m = 0xFF
    a, b, c = 0xF0, 0xCC, 0xAA
    assert s == (a ^ b ^ c) & m
    assert k == ((a & b) | (a & c) | (b & c)) & m


def test_csa15_counts_every_combination(src):
    adders = _adders(_body(src, "csa15"))
    assert len(adders) == 11
    n, size = 15, 1 << 15
    mask = (1 << size) - 1
    ins = _input_patterns(n)
    env = {f"v[{i}]": ins[i] for i in range(n)}
    env, depth = _simulate(adders, env, mask, _lut(src, "lop3_parity"), _lut(src, "lop3_majority"))
    want = _popcounts(ins, size)
    got = [env["p.a1"], env["p.a2"], env["p.a4"], env["p.a8"]]
    assert got == want[:4] and not any(want[4:])
    assert max(depth[k] for k in ("p.a1", "p.a2", "p.a4", "p.a8")) == 5


def test_csa16_plus_4_counts_every_combination(src):
    adders = _adders(_body(src, "csa16"))
    assert len(adders) == 15
    n, size = 20, 1 << 20
    mask = (1 << size) - 1
    ins = _input_patterns(n)
    env = {f"v[{i}]": ins[i] for i in range(16)}
    planes = {"p.a1": ins[16], "p.a2": ins[17], "p.a4": ins[18], "p.a8": ins[19]}
    env.update(planes)
    env, _ = _simulate(adders, env, mask, _lut(src, "lop3_parity"), _lut(src, "lop3_majority"))
    # the value on the left: a1 + 2 a2 + 4 a4 + 8 a8 + sum(v), as bit planes
    terms = list(ins[:16]) + [ins[16]] + [ins[17]] * 2 + [ins[18]] * 4 + [ins[19]] * 8
    want = _popcounts(terms, size)
    a16 = re.search(r"return (\w+);", _body(src, "csa16")).group(1)
    got = [env["p.a1"], env["p.a2"], env["p.a4"], env["p.a8"], env[a16]]
    assert got == want[:5] and not any(want[5:])


def test_the_planted_miswiring_is_caught(src):
    """A copy of CSA_15 with two inputs of one adder swapped for a carry
    fails the simulation (the check is not vacuous)."""
    adders = _adders(_body(src, "csa15"))
    s, k, a, b, c = adders[5]
    bad = list(adders)
    bad[5] = (s, k, a, b, "c0")           # feed a carry where a sum belongs
    n, size = 15, 1 << 15
    mask = (1 << size) - 1
    ins = _input_patterns(n)
    env = {f"v[{i}]": ins[i] for i in range(n)}
    env, _ = _simulate(bad, env, mask, _lut(src, "lop3_parity"), _lut(src, "lop3_majority"))
    want = _popcounts(ins, size)
    assert [env["p.a1"], env["p.a2"], env["p.a4"], env["p.a8"]] != want[:4]
