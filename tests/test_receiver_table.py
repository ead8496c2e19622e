"""Host logic of the receiver table (no GPU): a host program compiled with
nvcc from the library's own source builds the table every sweep path uses
(single grid, allocation-free, served shots), and it is compared with the
table's definition restated here.

Receiver r at (x, y, z) belongs to tile (y // ty) * ceil(nx / tx) + x // tx
at local index (y % ty) * tx + x % tx; the entries {z, local, r, tile} are
sorted by (tile, z, r) and start[t] is the number of entries of the tiles
before t. A receiver outside the interior makes the call fail (-1).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("rt") / "receiver_table")
    subprocess.run([nvcc, "-std=c++17", "-O2",
                    os.path.join(ROOT, "tests", "host", "receiver_table.cu"), "-o", exe],
                   check=True, capture_output=True)

    def run(dims, tile, rec):
        nx, ny, nz = dims
        text = "%d %d %d %d %d %d\n" % (nx, ny, nz, tile[0], tile[1], len(rec))
        text += "".join("%d %d %d\n" % tuple(r) for r in rec)
        out = subprocess.run([exe], input=text, capture_output=True, text=True,
                             check=True).stdout.split("\n")
        st = int(out[0])
        if st != 0:
            return st, None, None
        n = len(rec)
        ent = [tuple(int(v) for v in l.split()) for l in out[1:1 + n]]
        start = [int(l) for l in out[1 + n:] if l.strip()]
        return st, ent, start
    return run


def definition(dims, tile, rec):
    nx, ny, nz = dims
    tx, ty = tile
    ntx, nty = -(-nx // tx), -(-ny // ty)
    ent = []
    for r, (x, y, z) in enumerate(rec):
        ent.append((z, (y % ty) * tx + x % tx, r, (y // ty) * ntx + x // tx))
    ent.sort(key=lambda e: (e[3], e[0], e[2]))
    counts = np.bincount([e[3] for e in ent], minlength=ntx * nty)
    return ent, [0] + list(np.cumsum(counts))


@pytest.mark.parametrize("dims,tile,n,seed", [
    ((45, 38, 29), (32, 16), 500, 0),
    ((1024, 1024, 512), (32, 16), 4000, 1),
    ((200, 90, 300), (64, 8), 3000, 2),
    ((7, 5, 3), (32, 16), 40, 3),
    ((64, 64, 64), (64, 16), 0, 4),
])
def test_table_matches_its_definition(driver, dims, tile, n, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    rec = np.stack([rng.integers(0, nx, n), rng.integers(0, ny, n), rng.integers(0, nz, n)],
                   axis=1).tolist()
    # repeated receivers and every tile corner and edge
    rec += rec[: n // 10]
    for x in sorted({0, nx - 1} | set(range(tile[0] - 1, nx, tile[0])) | set(range(0, nx, tile[0]))):
        for y in sorted({0, ny - 1} | set(range(tile[1] - 1, ny, tile[1]))):
            rec.append([x, y, (x + y) % nz])
    st, ent, start = driver(dims, tile, rec)
    want_ent, want_start = definition(dims, tile, rec)
    assert st == 0
    assert ent == want_ent
    assert start == [int(v) for v in want_start]


@pytest.mark.parametrize("bad", [(-1, 0, 0), (45, 0, 0), (0, 38, 0), (0, 0, 29), (0, -3, 5)])
def test_receiver_outside_the_grid_is_refused(driver, bad):
    st, _, _ = driver((45, 38, 29), (32, 16), [[1, 2, 3], list(bad), [4, 5, 6]])
    assert st == -1
