"""Writes qs_ct_asm.inc: the Clifford+T op loop of the complex64 fused pass
(32 register slots, 5 register bits) as inline PTX with an indexed branch.

The interpreter stages every op of a Clifford+T pass as one byte code from a
dense range (see exec_ct / ct_code in qs_fused.cu):

    C_H  + j   (0..4)    H on register bit j (deferred 1/sqrt2)
    C_XH + j   (5..9)    X^1/2 on register bit j
    C_YH + j   (10..14)  Y^1/2 on register bit j
    C_T  + j   (15..19)  T phase on the slots with bit j set
    C_CZ + p   (20..29)  sign on the slots with both bits of pair p set
    C_CZO + j  (30..34)  sign on the slots with bit j set where the op's
                         selection outside the register set holds
    C_Z  + j   (35..39)  sign on the slots with bit j set

A C++ switch over these codes compiles to a tree of compares and branches
(about ten branches per op); here every case ends with its own copy of the
dispatch (threaded code): the next op's code, loaded while the case ran,
picks the next case by one indexed branch (brx.idx), and the code after it
is loaded in turn.  Every case does exactly the
arithmetic of the C++ cases (the same operations in the same order, packed
FP32x2 where both components see the same operation), so results are the
same bit for bit.

Run `python gen_ct_asm.py` in this directory after changing the op set; the
generated file is committed.
"""
import os

NS = 32          # register slots per thread
RB = 5           # register bits
NCODES = 40
C_H, C_XH, C_YH, C_T, C_CZ, C_CZO, C_Z = 0, 5, 10, 15, 20, 30, 35
F_C = "0f3F3504F3"       # 1/sqrt2 rounded to FP32
F_2C = "0f3FB504F3"      # 2 * that (exact)
F_NC = "0fBF3504F3"      # -(1/sqrt2)
F_2 = "0f40000000"
F_M1 = "0fBF800000"
F_P1 = "0f3F800000"


def pair_index(j, k):
    return j * 4 - (j * (j + 1)) // 2 + (k - 1)


def slot(s):
    return "%%%d" % s


def case_h(j):
    out = []
    for s in range(NS):
        if s & (1 << j):
            continue
        t = s | (1 << j)
        # x = x + y; y = y * (-2) + x
        out.append("add.rn.f32x2 %s, %s, %s;" % (slot(s), slot(s), slot(t)))
        out.append("fma.rn.f32x2 %s, %s, qM2, %s;" % (slot(t), slot(t), slot(s)))
    return out


def case_yh(j):
    out = []
    for s in range(NS):
        if s & (1 << j):
            continue
        t = s | (1 << j)
        # x = y * (-1) + x; y = y * 2 + x
        out.append("fma.rn.f32x2 %s, %s, qM1, %s;" % (slot(s), slot(t), slot(s)))
        out.append("fma.rn.f32x2 %s, %s, qP2, %s;" % (slot(t), slot(t), slot(s)))
    return out


def case_xh(j):
    out = []
    for s in range(NS):
        if s & (1 << j):
            continue
        t = s | (1 << j)
        # x.re = x.re + y.im; y.im = y.im * 2 - x.re;
        # x.im = x.im - y.re; y.re = y.re * 2 + x.im
        out += ["mov.b64 {xr, xi}, %s;" % slot(s),
                "mov.b64 {yr, yi}, %s;" % slot(t),
                "add.rn.f32 xr, xr, yi;",
                "neg.f32 tn, xr;",
                "fma.rn.f32 yi, yi, %s, tn;" % F_2,
                "sub.rn.f32 xi, xi, yr;",
                "fma.rn.f32 yr, yr, %s, xi;" % F_2,
                "mov.b64 %s, {xr, xi};" % slot(s),
                "mov.b64 %s, {yr, yi};" % slot(t)]
    return out


def case_t(j):
    out = []
    for s in range(NS):
        if not s & (1 << j):
            continue
        # re = re * c; re = im * (-c) + re; im = im * 2c + re
        out += ["mov.b64 {xr, xi}, %s;" % slot(s),
                "mul.rn.f32 xr, xr, %s;" % F_C,
                "fma.rn.f32 xr, xi, %s, xr;" % F_NC,
                "fma.rn.f32 xi, xi, %s, xr;" % F_2C,
                "mov.b64 %s, {xr, xi};" % slot(s)]
    return out


def case_sign(mask, factor):
    return ["mul.rn.f32x2 %s, %s, %s;" % (slot(s), slot(s), factor)
            for s in range(NS) if (s & mask) == mask]


def case_czo(j):
    # the selection outside the register set: (idx & qmask) == qmask, the
    # op's qmask at byte 8 of its 16-byte staged record (op qo - 1: the
    # dispatch has already advanced qo)
    return ["mad.lo.u32 qa, qo, 16, qmb;",
            "ld.shared.u64 qm, [qa];",
            "and.b64 qt, %36, qm;",
            "setp.eq.u64 qp, qt, qm;",
            "selp.f32 qsg, %s, %s, qp;" % (F_M1, F_P1),
            "mov.b64 qS, {qsg, qsg};"] + case_sign(1 << j, "qS")


def cases():
    body = [None] * NCODES
    for j in range(RB):
        body[C_H + j] = case_h(j)
        body[C_XH + j] = case_xh(j)
        body[C_YH + j] = case_yh(j)
        body[C_T + j] = case_t(j)
        body[C_CZO + j] = case_czo(j)
        body[C_Z + j] = case_sign(1 << j, "qM1")
    for j in range(RB):
        for k in range(j + 1, RB):
            body[C_CZ + pair_index(j, k)] = case_sign((1 << j) | (1 << k), "qM1")
    assert all(b is not None for b in body)
    return body


def dispatch(L):
    """Runs op qo (its code in qcn, loaded earlier): leaves when qo reaches
    the end, loads op qo + 1's code (the staged codes run past the last op),
    and branches to op qo's case; a code outside the table is clamped to the
    extra entry, which only dispatches the next op (the staging never makes
    one)."""
    return ["setp.ge.s32 qp, qo, %35;",
            "@qp bra.uni " + L("DONE") + ";",
            "min.u32 qc, qcn, %d;" % NCODES,
            "add.u32 qo, qo, 1;",
            "add.u32 qa, %32, qo;",
            "ld.shared.u8 qcn, [qa];",
            "brx.idx.uni qc, " + L("TBL") + ";"]


def asm_text(prefix):
    """PTX of the loop over ops [%34, %35): %0..%31 the slots (re in the low
    word, im in the high word), %32 the shared address of the byte codes,
    %33 that of the first op record's qmask, %36 the thread's qubit index
    bits."""
    L = lambda name: "%s_%s" % (prefix, name)
    lines = ["{",
             ".reg .pred qp;",
             ".reg .u32 qo, qc, qcn, qa, qmb;",
             ".reg .b64 qm, qt, qS, qM2, qM1, qP2;",
             ".reg .f32 xr, xi, yr, yi, tn, qsg;",
             "mov.b64 qM2, {0fC0000000, 0fC0000000};",
             "mov.b64 qM1, {%s, %s};" % (F_M1, F_M1),
             "mov.b64 qP2, {%s, %s};" % (F_2, F_2),
             "sub.u32 qmb, %33, 16;",
             "mov.u32 qo, %34;",
             "add.u32 qa, %32, qo;",
             "ld.shared.u8 qcn, [qa];",
             L("TBL") + ": .branchtargets " + ", ".join([L("C%d" % c) for c in range(NCODES)] + [L("NEXT")]) + ";",
             L("NEXT") + ":"]
    lines += dispatch(L)
    for c, b in enumerate(cases()):
        lines.append(L("C%d" % c) + ":")
        lines += b
        lines += dispatch(L)
    lines += [L("DONE") + ":", "}"]
    return lines


def emit():
    out = ["// qs_ct_asm.inc -- generated by gen_ct_asm.py (same directory); do not edit.",
           "//",
           "// The Clifford+T op loop of the complex64 fused pass (32 slots, 5",
           "// register bits) as inline PTX: one byte-code load and one indexed",
           "// branch per op.  CtAsm<0> and CtAsm<1> differ only in their labels, so",
           "// that one kernel can hold two inlined copies.",
           "",
           "template <int VARIANT> struct CtAsm;"]
    for v, prefix in enumerate(("QSCTA", "QSCTB")):
        out.append("template <> struct CtAsm<%d> {" % v)
        out.append("    static __device__ __forceinline__ void run(unsigned long long (&u)[32], uint32_t codes,")
        out.append("                                               uint32_t qmask0, int ob, int ub,")
        out.append("                                               unsigned long long idx)")
        out.append("    {")
        out.append("        asm volatile(")
        for line in asm_text(prefix):
            out.append('            "%s\\n"' % line)
        ops = ", ".join('"+l"(u[%d])' % s for s in range(NS))
        out.append("            : " + ops)
        out.append('            : "r"(codes), "r"(qmask0), "r"(ob), "r"(ub), "l"(idx)')
        out.append('            : "memory");')
        out.append("    }")
        out.append("};")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "qs_ct_asm.inc"), "w") as f:
        f.write(emit())
