"""Index arithmetic of the wavelet kernels (csrc/wavelet.cu), emulated on the CPU:
every element a CTA stages lies inside its level's block, and the staged window
holds, at the periodic positions, every input that a kept output reads.

The tile constants are read from the source, so the emulation follows the
kernels.  The coarse levels of small images have windows that span their block
more than once: a single conditional wrap would index past it there."""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2108_01438_gb300", "csrc", "wavelet.cu")


def _tiles():
    s = open(SRC).read()
    fwd = re.search(r"struct FwdTile \{\s*static constexpr int TA = (\d+), TB = SMALL \? (\d+) : (\d+);", s)
    inv = re.search(r"struct InvTile \{\s*static constexpr int TR = (\d+), TC = SMALL \? (\d+) : (\d+);", s)
    assert fwd and inv, "tile constants not found in wavelet.cu"
    ta, tb_small, tb_big = map(int, fwd.groups())
    tr, tc_small, tc_big = map(int, inv.groups())
    return {True: (ta, tb_small), False: (ta, tb_big)}, {True: (tr, tc_small), False: (tr, tc_big)}


FWD, INV = _tiles()


def _wrap_down(v, n):
    while v >= n:          # the kernels' wrap
        v -= n
    return v


def _analysis_wrap(v, n, small_block):
    """The analysis kernel's wrap: one subtraction, and the remainder when the
    block is smaller than the window."""
    if v >= n:
        v -= n
    return v % n if small_block else v


def _analysis_ok(P, N, small):
    """dwt_fwd_kernel: a tile of TA x TB coefficients per band stages the
    (2 TA + 6) x (2 TB + 6) input window at (2 a0, 2 b0)."""
    ta, tb = FWD[small]
    rows, cols = 2 * ta + 6, 2 * tb + 6
    Ph, Nh = P // 2, N // 2
    small_block = P < rows or N < cols
    for a0 in range(0, Ph, ta):
        for b0 in range(0, Nh, tb):
            staged = {}
            for i in range(rows):
                for j in range(cols):
                    r = _analysis_wrap(2 * a0 + i, P, small_block)
                    c = _analysis_wrap(2 * b0 + j, N, small_block)
                    assert 0 <= r < P and 0 <= c < N
                    staged[(i, j)] = (r, c)
            # kept outputs (A < Ph, B < Nh) read window rows 2(A - a0) + t, t < 8
            for A in range(a0, min(a0 + ta, Ph)):
                for t in range(8):
                    i = 2 * (A - a0) + t
                    assert i < rows and staged[(i, 0)][0] == (2 * A + t) % P
            for B in range(b0, min(b0 + tb, Nh)):
                for t in range(8):
                    j = 2 * (B - b0) + t
                    assert j < cols and staged[(0, j)][1] == (2 * B + t) % N


def _synthesis_ok(P, N, small):
    """dwt_inv_kernel: a TR x TC output tile stages (TR/2 + 3) x (TC/2 + 3)
    coefficients per band from (r0/2 - 3, c0/2 - 3)."""
    tr, tc = INV[small]
    rows, cols = tr // 2 + 3, tc // 2 + 3
    Ph, Nh = P // 2, N // 2
    for r0 in range(0, P, tr):
        for c0 in range(0, N, tc):
            for ia in range(rows):
                A = r0 // 2 - 3 + ia
                if A < 0:
                    A += Ph
                A = _wrap_down(A, Ph)
                assert 0 <= A < Ph and A == (r0 // 2 - 3 + ia) % Ph
            for ib in range(cols):
                B = c0 // 2 - 3 + ib
                if B < 0:
                    B += Nh
                B = _wrap_down(B, Nh)
                assert 0 <= B < Nh and B == (c0 // 2 - 3 + ib) % Nh


def _levels(nx, nz):
    P, N = nx, nz
    for lev in range(3):
        yield P, N, lev > 0
        P //= 2
        N //= 2


@pytest.mark.parametrize("nx,nz", [(32, 32), (32, 64), (40, 48), (64, 256), (96, 72), (128, 40), (256, 512)])
def test_wavelet_windows_stay_inside_their_blocks(nx, nz):
    for P, N, small in _levels(nx, nz):
        _analysis_ok(P, N, small)
        _synthesis_ok(P, N, small)


def test_kernels_use_the_emulated_wrap():
    s = open(SRC).read()
    for stmt in ("if (row >= P) row -= P;", "if (col >= N) col -= N;", "row %= P;", "col %= N;",
                 "if (P < kRows || N < kCols) stage(std::true_type());",
                 "while (A >= Ph) A -= Ph;", "while (Bc >= Nh) Bc -= Nh;"):
        assert stmt in s, stmt


def test_single_wrap_would_leave_the_block_at_small_sizes():
    """The case the remainder exists for: level 3 of a 32-row image has an 8-row
    block and a 38-row window."""
    ta, _ = FWD[True]
    rows, P = 2 * ta + 6, 32 >> 2
    once = [(i - P if i >= P else i) for i in range(rows)]
    assert max(once) >= P

