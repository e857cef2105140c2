"""Row chunking of the split-m Gram kernels (paper_1703_06303_gb300/csrc/wlr_plan.h),
compiled on the host and checked against a restatement of its rule: the chunk count that
minimises (waves) x (rows per chunk + 128), waves = ceil(tiles x chunks / slots), taking
the fewest chunks within 3% of that minimum; rows a multiple of 32 covering m."""
import itertools
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cdiv(a, b):
    return -(-a // b)


def _rule(m, tiles, slots):
    cand = []
    for n in range(1, max(1, min(128, _cdiv(m, 32))) + 1):
        rows = max(32, _cdiv(_cdiv(m, n), 32) * 32)
        nn = _cdiv(m, rows)
        cand.append((nn, rows, _cdiv(tiles * nn, slots) * (rows + 128)))
    best = min(c[2] for c in cand)
    ok = [c for c in cand if c[2] * 100 <= best * 103]
    return min(ok, key=lambda c: (c[0], c[2]))


@pytest.fixture(scope="module")
def plan_bin(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("plan") / "plan_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1703_06303_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "plan_check.cpp"), "-o", out], check=True)
    return out


def _run(binary, triples):
    inp = "".join(f"{m} {t} {s}\n" for m, t, s in triples)
    r = subprocess.run([binary], input=inp, capture_output=True, text=True, check=True)
    return [tuple(map(int, line.split())) for line in r.stdout.strip().splitlines()]


def test_whole_wave_chunking_matches_the_rule(plan_bin):
    ms = [32, 100, 1200, 4800, 19200, 76800, 300000]
    tiles = [1, 2, 4, 9, 12, 25, 64]
    slots = [152, 304]
    rows = _run(plan_bin, list(itertools.product(ms, tiles, slots)))
    for m, t, s, nch, r, cn, cr in rows:
        assert r % 32 == 0 and nch * r >= m and (nch - 1) * r < m
        best = _rule(m, t, s)
        assert (nch, r) == best[:2], (m, t, s, nch, r, best)
        assert cr % 32 == 0 and cn * cr >= m and 1 <= cn <= 128


def test_the_launches_measured_on_gb300(plan_bin):
    # (m, tiles) of the tensor-core Grams on 152 SMs, one CTA per SM: the per-iteration
    # Q1^T [Q1 A2] at 19200 x 400 and 76800 x 1000, K at both sizes
    got = {(m, t): (n, r) for m, t, _, n, r, _, _ in
           _run(plan_bin, [(19200, 4, 152), (76800, 9, 152), (19200, 12, 152), (76800, 64, 152)])}
    assert got[(19200, 4)] == (38, 512)      # 152 CTAs, one wave
    assert got[(76800, 9)] == (16, 4800)     # 144 CTAs instead of 153 (a second wave)
    assert got[(19200, 12)] == (12, 1600)    # 144 CTAs instead of 156
    assert got[(76800, 64)] == (7, 10976)    # 448 CTAs, three whole waves
