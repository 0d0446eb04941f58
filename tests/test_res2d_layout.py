"""The resident 2D kernel's slab layout against the reads of its stencil (host logic, no GPU).

The kernel (csrc/micro_fp32_2d.cuh) holds each box slab of S interior rows in shared
memory as consecutive arrays: the states vA, vB (and vC for RK4P), 3 components of
S + 2r rows of stride LD each; the x-face coefficients afx (S + 3 or S + 1 rows of
stride LDI); the y-face coefficients afy (S rows of stride LDY); then m_init,
H(m_init) and H(W) (stride LDI) and, for RK4P, the stage accumulator. Thread t of a
box owns the tile of TR rows starting at ii0 = (t / CPp) TR and the column pair
jj0 = 2 (t mod CPp). The stencil reads its rows without clamping, so the tiles of a
ragged last tile row read up to TR - 1 rows past the slab; the layout places the
arrays that can overrun first and pads the slab so that those reads stay inside it.
Where a row group of 16 or 32 tiles leaves two spare lanes (res_yshfl_ok), every
lane of the box's warps runs the stencil on clamped indices.

This test restates the layout rule (strides, offsets, padding) and the stencil's
read and write pattern, and checks for every compiled instance (parsed from the
res2d_*.cu sources), every box size it can hold, every cluster size up to 8 and
every slab of the split, that every read stays inside the slab's allocation and
every write inside its own array.
"""
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2108_09463_gb300", "csrc")
MAX_CLUSTER = 8
MAX_BOX_STRIDE_N = 160      # the largest box the box-stride instances are planned for


def _header_int(name):
    src = open(os.path.join(CSRC, "micro_fp32_2d.cuh")).read()
    return int(re.search(r"constexpr int %s = (\d+);" % name, src).group(1))


K_TR = _header_int("kResTR")


def cp_pad(Ni):
    CP = (Ni + 1) // 2
    if CP <= 16:
        return 16
    if 28 < CP <= 32:
        return 32
    return (CP + 3) & ~3


def stride(minimum, CPp):
    if CPp in (16, 32):
        return (minimum + 1) & ~1
    r = (CPp // 2) & 7
    s = minimum
    while (s & 7) != r:
        s += 1
    return s


def dims(N, R, S, TR, rk4):
    Ni = N - 2 * R
    CPp = cp_pad(Ni)
    return dict(N=N, Ni=Ni, S=S, rows=S + 2 * R, CPp=CPp, LD=stride(N + 4, CPp), LDI=stride(Ni, CPp),
                nf=S + (3 if R == 3 else 1), LDY=stride(Ni + (4 if R == 3 else 2), CPp), TR=TR, rk4=rk4)


def offsets(d, pad=True):
    o, x, need = {}, 0, 0
    over = ((d["S"] + d["TR"] - 1) // d["TR"]) * d["TR"] - d["S"] + 1

    def place(name, size, st):
        nonlocal x, need
        o[name] = (x, size)
        x += size
        if st > 0:
            need = max(need, x + over * st + 8)

    place("vA", 3 * d["rows"] * d["LD"], d["LD"])
    place("vB", 3 * d["rows"] * d["LD"], d["LD"])
    if d["rk4"]:
        place("vC", 3 * d["rows"] * d["LD"], d["LD"])
    place("afx", d["nf"] * d["LDI"], d["LDI"])
    place("afy", d["S"] * d["LDY"], d["LDY"])
    place("mi", 3 * d["S"] * d["LDI"], 0)
    place("hi", 3 * d["S"] * d["LDI"], 0)
    place("hw", d["S"] * d["LDI"], 0)
    if d["rk4"]:
        place("acc", 3 * d["TR"] * 2 * (((d["S"] + d["TR"] - 1) // d["TR"]) * d["CPp"]), 0)
    return o, ((max(x, need) if pad else x) + 3) & ~3


def instances():
    """(R, NC, SAC, TR, stepper) of every compiled 2D instance."""
    pat = re.compile(r"\{(\d+), (\d+), (\d+), (\d+), micro_fp32_2d_kernel<(\d+), (kResTR|\d+), (\d+), (\d+)(?:, (\d+))?>")
    out = set()
    for f in sorted(os.listdir(CSRC)):
        if f.startswith("res2d_") and f.endswith(".cu"):
            for m in pat.finditer(open(os.path.join(CSRC, f)).read()):
                R, NC, SAC = int(m.group(5)), int(m.group(7)), int(m.group(8))
                TR = K_TR if m.group(6) == "kResTR" else int(m.group(6))
                out.add((R, NC, SAC, TR, int(m.group(9) or 0)))
    return sorted(out)


def slabs(R, NC, SAC):
    """(N, Sa, S) of every slab the instance can be given: N <= NC with Sa <= SAC for a
    canvas, any N up to the planning limit for the box-stride instance."""
    nmax = NC if NC > 0 else MAX_BOX_STRIDE_N
    for N in range(2 * R + 2, nmax + 1):
        Ni = N - 2 * R
        for cs in range(1, MAX_CLUSTER + 1):
            Sa = Ni if cs == 1 else (Ni + cs - 1) // cs
            if NC > 0 and Sa > SAC:
                continue
            for rank in range(cs):
                S = max(0, min(Sa, Ni - rank * Sa))
                if S > 0:
                    yield N, Sa, S


def check_slab(R, NC, SAC, TR, st, N, Sa, S, pad=True):
    """First violation (a string) of the slab's reads and writes, or None. pad=False
    drops the layout's padding (to show that the check can fail). Every thread's
    reads are the offsets below; their least and greatest values per thread bound
    them (offsets grow with the row and the column)."""
    d = dims(NC, R, SAC, TR, st) if NC > 0 else dims(N, R, Sa, TR, st)
    o, total = offsets(d, pad)
    Ni, CPp, LD, LDI, LDY, rows = N - 2 * R, d["CPp"], d["LD"], d["LDI"], d["LDY"], d["rows"]
    ntile = ((S + TR - 1) // TR) * CPp
    yshfl = CPp in (16, 32) and (Ni + 1) // 2 <= CPp - 2
    nthreads = ((ntile + 31) // 32) * 32 if yshfl else ntile
    t = np.arange(nthreads)
    ii0, jj0 = (t // CPp) * TR, 2 * (t % CPp)
    active = (t < ntile) & (jj0 < Ni)
    if yshfl:
        jj0 = np.minimum(jj0, 2 * ((Ni + 1) // 2) + (2 if R == 3 else 0))
        ii0 = np.minimum(ii0, ((S + TR - 1) // TR - 1) * TR)
        run = np.ones(nthreads, bool)
    else:
        run = active
    ii0, jj0, act = ii0[run], jj0[run], active[run]
    j0 = R + jj0
    states = ["vA", "vB"] + (["vC"] if st else [])
    # column offsets from j0 + 1 in a state row: x direction (0, 1) on rows ii0 .. ii0 + TR + 2R - 1,
    # y direction on rows ii0 + R .. ii0 + R + TR - 1
    ycols = (-3, -1) if (yshfl and R == 3) else ((-1, -1) if yshfl else ((-4, 4) if R == 3 else (-2, 3)))
    lo_state = np.minimum(ii0 * LD + j0 + 1, (ii0 + R) * LD + j0 + 1 + ycols[0])
    hi_state = np.maximum((ii0 + TR + 2 * R - 1) * LD + j0 + 2, (ii0 + R + TR - 1) * LD + j0 + 1 + ycols[1])
    spans = [(o[arr][0] + lo_state, o[arr][0] + 2 * rows * LD + hi_state, arr) for arr in states]
    nfr = TR + (3 if R == 3 else 1)
    spans.append((o["afx"][0] + ii0 * LDI + jj0, o["afx"][0] + (ii0 + nfr - 1) * LDI + jj0 + 1, "afx"))
    yhi = 1 if yshfl else (4 if R == 3 else 2)
    spans.append((o["afy"][0] + ii0 * LDY + jj0, o["afy"][0] + (ii0 + TR - 1) * LDY + jj0 + yhi, "afy"))
    for lo, hi, arr in spans:
        if len(lo) and (lo.min() < 0 or hi.max() >= total):
            k = int(np.argmax(hi)) if hi.max() >= total else int(np.argmin(lo))
            return f"{arr} read of tile ({ii0[k]}, {jj0[k]}) outside [0, {total}): {lo[k]} .. {hi[k]}"
    # the update: own nodes of the tile rows inside the slab, inside their own arrays
    ii0a, j0a, jj0a = ii0[act], j0[act], jj0[act]
    for tt in range(TR):
        ii = ii0a + tt
        m = ii < S
        if not m.any():
            continue
        for arr in states:
            w = 2 * rows * LD + (ii[m] + R) * LD + j0a[m] + 2
            if w.max() >= o[arr][1] or ((ii[m] + R) * LD + j0a[m] + 1).min() < 0:
                return f"write of {arr} outside its {o[arr][1]} floats"
        for arr, ncomp in (("mi", 3), ("hi", 3), ("hw", 1)):
            r = (ncomp - 1) * d["S"] * LDI + ii[m] * LDI + jj0a[m] + 1
            if r.max() >= o[arr][1]:
                return f"{arr} access outside its {o[arr][1]} floats"
    return None


INSTANCES = instances()


def test_instances_parsed():
    # the packs, the cluster canvases, the 2-row canvases, the box-stride and the RK4P instances
    assert len(INSTANCES) >= 24
    assert any(NC == 0 for _, NC, _, _, _ in INSTANCES)
    assert any(st == 1 for *_, st in INSTANCES)
    assert any(TR == 2 for _, _, _, TR, _ in INSTANCES)


@pytest.mark.parametrize("inst", INSTANCES, ids=lambda i: "R%d_NC%d_SAC%d_TR%d_st%d" % i)
def test_stencil_reads_stay_inside_the_slab(inst):
    R, NC, SAC, TR, st = inst
    n = 0
    for N, Sa, S in slabs(R, NC, SAC):
        err = check_slab(R, NC, SAC, TR, st, N, Sa, S)
        assert err is None, f"N={N} Sa={Sa} S={S}: {err}"
        n += 1
    assert n > 0


def test_the_check_sees_an_unpadded_slab():
    """Without the padding some ragged slab reads past its end: the box-stride instance
    (strides from the box) on boxes whose last tile row is ragged."""
    fails = [(N, Sa, S) for N, Sa, S in slabs(3, 0, 0)
             if check_slab(3, 0, 0, K_TR, 0, N, Sa, S, pad=False) is not None]
    assert fails
