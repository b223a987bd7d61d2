"""The Clifford+T op loop in inline PTX (csrc/qs_ct_asm.inc, written by
csrc/gen_ct_asm.py): the committed file is the generator's output, and every
case body, run by a small interpreter of the instruction forms it uses
(FP32 arithmetic in numpy, FMA rounded once), applies the gate of its byte
code to the right slots:

    H        x' = x + y,      y' = x - y        (1/sqrt2 deferred)
    X^1/2    x' = x - i y,    y' = y - i x      (1/sqrt2 deferred)
    Y^1/2    x' = x - y,      y' = x + y        (1/sqrt2 deferred)
    T        slots with the bit set times e^{i pi/4}
    CZ       slots with both bits set negated
    CZ (one register bit, selection outside the register set)
             slots with the bit set negated when (idx & qmask) == qmask
    Z        slots with the bit set negated

x is the slot with the register bit clear and y its partner (Sec. "Random
circuits" gate set; the deferred factor is applied once per pass)."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1608_00263_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_ct_asm", os.path.join(CSRC, "gen_ct_asm.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    return g


def test_generated_file_is_current():
    with open(os.path.join(CSRC, "qs_ct_asm.inc")) as f:
        assert f.read() == _gen().emit()


f32 = np.float32


def _imm(tok):
    assert tok.startswith("0f")
    return np.frombuffer(int(tok[2:], 16).to_bytes(4, "little"), dtype=np.float32)[0]


def _fma(a, b, c):
    # FP32 fused multiply-add: the product is exact in FP64, one rounding
    # to FP32 of the FP64 sum (a double rounding only when the FP64 sum
    # itself rounds, far below the tolerance used here)
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


class Machine:
    """Registers of one thread: %k (k < 32) are the slots as (re, im) FP32
    pairs; the op runs as op 0 (qo = 1 after the dispatch, its qmask at
    byte 8 of the op records); %36 the index bits."""

    def __init__(self, slots, idx, qmask):
        self.r = {"%%%d" % s: [f32(v.real), f32(v.imag)] for s, v in enumerate(slots)}
        self.r["qo"] = 1
        self.r["qmb"] = 8 - 16
        self.qmask = qmask
        self.r["%36"] = idx
        self.r["qM2"] = [f32(-2), f32(-2)]
        self.r["qM1"] = [f32(-1), f32(-1)]
        self.r["qP2"] = [f32(2), f32(2)]

    def val(self, tok):
        return _imm(tok) if tok.startswith("0f") else self.r[tok]

    def run(self, lines):
        for line in lines:
            op, rest = line.rstrip(";").split(None, 1)
            args = [a.strip() for a in rest.replace("{", "").replace("}", "").split(",")]
            r = self.r
            if op == "add.rn.f32x2":
                a, b = r[args[1]], r[args[2]]
                r[args[0]] = [f32(a[0] + b[0]), f32(a[1] + b[1])]
            elif op == "fma.rn.f32x2":
                a, b, c = r[args[1]], r[args[2]], r[args[3]]
                r[args[0]] = [_fma(a[0], b[0], c[0]), _fma(a[1], b[1], c[1])]
            elif op == "mul.rn.f32x2":
                a, b = r[args[1]], r[args[2]]
                r[args[0]] = [f32(a[0] * b[0]), f32(a[1] * b[1])]
            elif op == "mov.b64":
                if line.split(None, 1)[1].startswith("{"):      # unpack
                    lo, hi, src = args
                    r[lo], r[hi] = r[src]
                else:                                            # pack
                    dst, lo, hi = args
                    r[dst] = [r[lo], r[hi]]
            elif op == "add.rn.f32":
                r[args[0]] = f32(self.val(args[1]) + self.val(args[2]))
            elif op == "sub.rn.f32":
                r[args[0]] = f32(self.val(args[1]) - self.val(args[2]))
            elif op == "mul.rn.f32":
                r[args[0]] = f32(self.val(args[1]) * self.val(args[2]))
            elif op == "fma.rn.f32":
                r[args[0]] = _fma(self.val(args[1]), self.val(args[2]), self.val(args[3]))
            elif op == "neg.f32":
                r[args[0]] = f32(-self.val(args[1]))
            elif op == "mad.lo.u32":
                r[args[0]] = r[args[1]] * int(args[2]) + r[args[3]]
            elif op == "ld.shared.u64":
                assert args[1] == "[qa]" and r["qa"] == 8     # op 0's qmask
                r[args[0]] = self.qmask
            elif op == "and.b64":
                r[args[0]] = r[args[1]] & r[args[2]]
            elif op == "setp.eq.u64":
                r[args[0]] = r[args[1]] == r[args[2]]
            elif op == "selp.f32":
                r[args[0]] = _imm(args[1]) if r[args[3]] else _imm(args[2])
            else:
                raise AssertionError("instruction form not interpreted: " + line)
        return np.array([complex(*self.r["%%%d" % s]) for s in range(32)])


def _expected(code, slots, selected):
    g = _gen()
    a = slots.astype(np.complex128).copy()
    bit = lambda s, j: (s >> j) & 1
    w = np.exp(1j * np.pi / 4)
    if code < g.C_T:
        j = code % 5
        for s in range(32):
            if bit(s, j):
                continue
            x, y = a[s], a[s | 1 << j]
            if code < g.C_XH:
                a[s], a[s | 1 << j] = x + y, x - y
            elif code < g.C_YH:
                a[s], a[s | 1 << j] = x - 1j * y, y - 1j * x
            else:
                a[s], a[s | 1 << j] = x - y, x + y
    elif code < g.C_CZ:
        j = code - g.C_T
        for s in range(32):
            if bit(s, j):
                a[s] *= w
    elif code < g.C_CZO:
        pairs = [(j, k) for j in range(5) for k in range(j + 1, 5)]
        j, k = pairs[code - g.C_CZ]
        assert g.pair_index(j, k) == code - g.C_CZ
        for s in range(32):
            if bit(s, j) and bit(s, k):
                a[s] = -a[s]
    else:
        j = code - (g.C_CZO if code < g.C_Z else g.C_Z)
        if code >= g.C_Z or selected:
            for s in range(32):
                if bit(s, j):
                    a[s] = -a[s]
    return a


@pytest.mark.parametrize("code", range(40))
def test_each_case_applies_its_gate(code):
    g = _gen()
    body = g.cases()[code]
    rng = np.random.default_rng(code)
    slots = (rng.standard_normal(32) + 1j * rng.standard_normal(32)).astype(np.complex64)
    # selection outside the register set: met (idx has every qmask bit) and
    # not met (one bit missing)
    for idx, qmask, selected in ((0b1011 << 20, 0b0011 << 20, True), (0b1001 << 20, 0b0011 << 20, False)):
        got = Machine(slots, idx, qmask).run(body)
        want = _expected(code, slots, selected)
        assert np.max(np.abs(got - want)) <= 4e-6 * max(1.0, np.max(np.abs(want))), (code, selected)


def test_case_table_covers_every_code_once():
    g = _gen()
    text = "\n".join(g.asm_text("P"))
    labels = ["P_C%d:" % c for c in range(g.NCODES)]
    assert all(text.count(lab) == 1 for lab in labels)
    targets = [ln for ln in g.asm_text("P") if ".branchtargets" in ln]
    assert len(targets) == 1
    assert targets[0].split(".branchtargets")[1].strip(" ;").split(", ") == \
        ["P_C%d" % c for c in range(g.NCODES)] + ["P_NEXT"]
    # threaded dispatch: the entry and every case end in the same dispatch
    d = g.dispatch(lambda name: "P_" + name)
    assert text.count("\n".join(d)) == g.NCODES + 1
    assert text.count("brx.idx.uni") == g.NCODES + 1
