"""The cluster form's partition of a level into the blocks of a cluster's CTAs (cluster_partition in
csrc/ff_internal.h, used on the host to size a launch and on the device by every CTA), checked on the CPU
against a brute-force enumeration.  For every grid of up to 40 x 40 pixels and cluster of 1 to 16 CTAs, the rule
picks, among the divisor pairs bx x by = n that leave every block at least one pixel wide and high, the one with
the smallest total block perimeter (w * by + h * bx, the first such pair by bx on a tie), or reports that there
is none.  Every block of the partition fits in the ceil(w / bx) x ceil(h / by) extent that cluster_smem_bytes
reserves, the blocks tile the grid exactly, and the shared-memory size is the one that extent implies."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1805_03517_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "ff_internal.h"
int main() {
    for (int w = 1; w <= 40; w++)
        for (int h = 1; h <= 40; h++)
            for (int n = 1; n <= 16; n++) {
                int bx = -1, by = -1;
                const bool ok = ff::cluster_partition(w, h, n, bx, by);
                const unsigned long long smem = ok ? (unsigned long long)ff::cluster_smem_bytes(w, h, bx, by) : 0ull;
                std::printf("%d %d %d %d %d %d %llu\n", w, h, n, ok ? 1 : 0, ok ? bx : 0, ok ? by : 0, smem);
            }
    return 0;
}
"""


def expected_partition(w, h, n):
    best = None
    for a in range(1, n + 1):
        if n % a:
            continue
        b = n // a
        if a > w or b > h:
            continue
        score = w * b + h * a
        if best is None or score < best[0]:
            best = (score, a, b)
    return None if best is None else best[1:]


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("partition")
    src, exe = d / "partition.cu", d / "partition"
    src.write_text(PROGRAM)
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I",
                        CSRC, "-o", str(exe), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return [tuple(int(v) for v in line.split()) for line in out.splitlines()]


def test_partition_is_the_smallest_perimeter_divisor_pair(rows):
    assert len(rows) == 40 * 40 * 16
    for w, h, n, ok, bx, by, _ in rows:
        want = expected_partition(w, h, n)
        assert bool(ok) == (want is not None), (w, h, n)
        if ok:
            assert (bx, by) == want, (w, h, n, bx, by, want)


def test_blocks_tile_the_grid_within_the_reserved_extent(rows):
    for w, h, n, ok, bx, by, smem in rows:
        if not ok:
            continue
        mw, mh = -(-w // bx), -(-h // by)
        assert smem == 16 + 4 * (2 * mw + 2 * mh) + 8 * mw * mh, (w, h, n)
        covered = 0
        for j in range(by):
            y0, y1 = j * h // by, (j + 1) * h // by
            for i in range(bx):
                x0, x1 = i * w // bx, (i + 1) * w // bx
                assert 1 <= x1 - x0 <= mw and 1 <= y1 - y0 <= mh, (w, h, n, i, j)
                covered += (x1 - x0) * (y1 - y0)
        assert covered == w * h, (w, h, n)
