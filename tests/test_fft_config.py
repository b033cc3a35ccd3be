"""Shape rules of the FFT tile table in csrc/fft.cuh, checked on the CPU.

The kernels index their registers, shared memory and global rows from the
table's radix split (R0, R1), elements per thread E, strided lines SB and x
pairs XP; an entry that breaks one of these rules would make a kernel read
or write outside its tile.  Every entry, default and alternative, is checked
here before any of it runs on a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2109_10375_gb300", "csrc")
SMEM_MAX = 227 * 1024


def _table():
    text = open(os.path.join(SRC, "fft.cuh")).read()
    pat = re.compile(r"template <> struct FftCfg<(\d+), (\d)>\s*\{\s*static constexpr int\s+"
                     r"R0 = (\d+),\s*R1 = (\d+),\s*E = (\d+),\s*SB = (\d+),\s*XP = (\d+);\s*\};")
    rows = [tuple(int(g) for g in m.groups()) for m in pat.finditer(text)]
    assert rows, "no FftCfg entries parsed"
    return rows


def test_every_size_has_a_default_and_the_dispatcher_knows_the_alternatives():
    rows = _table()
    sizes0 = sorted(n for n, v, *_ in rows if v == 0)
    assert sizes0 == [4, 8, 16, 32, 64, 128, 256, 512, 1024]
    alt = sorted(n for n, v, *_ in rows if v == 1)
    disp = open(os.path.join(SRC, "fft_f32.cu")).read()
    inst = sorted(int(n) for n in re.findall(r"radiation_field_n<float, (\d+), 1>", disp))
    assert inst == alt


@pytest.mark.parametrize("row", _table(), ids=lambda r: f"n{r[0]}v{r[1]}")
def test_tile_shape_rules(row):
    n, v, r0, r1, e, sb, xp = row
    # radix split and elements per thread
    assert r0 * r1 == n and r0 <= 32 and r1 <= 32
    assert e % r0 == 0 and (r1 == 1 or e % r1 == 0) and e >= r0 and e >= r1
    # threads of the strided and x passes: whole warps, at most 1024
    for lines in (sb, xp):
        assert (lines * n) % e == 0
        nt = lines * n // e
        assert nt % 32 == 0 and 32 <= nt <= 1024, (lines, nt)
    nt_x = xp * n // e
    assert (xp * (n // 2)) % nt_x == 0  # inverse x pass: equal loads per thread
    assert nt_x >= xp  # one thread per pair for the Nyquist column
    # shared memory, FP32 (FP64 for n <= 256 at twice the element size)
    for elem, real in ((8, 4), (16, 8)):
        if elem == 16 and (n > 256 or v != 0):
            continue
        pad = 8 if sb * elem == 64 else 0
        strided = (n * sb + (n // 32) * pad) * elem
        zpass = strided + (n // 2 + 1) * sb * real
        xpass = xp * (n + n // r0) * elem
        assert max(strided, zpass, xpass) <= SMEM_MAX, (strided, zpass, xpass)
