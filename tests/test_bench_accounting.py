"""The algorithmic byte counts behind the bench's roofline fractions, checked
against a per-line enumeration on small grids, and the traffic file's
source-hash check (a capture taken on other kernel sources is not reported).
"""
import pytest

import bench


def _enumerate_cpml(shape, npml, esize):
    """Bytes of one layered step counted line by line: the sweep's per-point
    bytes at every point; along each axis, every line has 2 (npml + 4)
    segment points (u^n, C, u^{n+1} read, u^{n+1} written) and 2 npml slab
    cells (psi, zeta read and written, FP32)."""
    nx, ny, nz = shape
    per_pt = 3 * esize + 4
    total = per_pt * nx * ny * nz
    w = npml + 4
    for n, nlines in ((nx, ny * nz), (ny, nx * nz), (nz, nx * ny)):
        for _ in range(nlines):
            seg = [i for i in range(n) if i < w or i >= n - w]
            slab = [i for i in range(n) if i < npml or i >= n - npml]
            total += per_pt * len(seg) + 16 * len(slab)
    return total


@pytest.mark.parametrize("shape,npml,esize", [((40, 36, 44), 8, 4), ((48, 40, 40), 16, 4),
                                              ((40, 36, 44), 8, 2), ((64, 48, 56), 16, 2)])
def test_cpml_bytes_per_step_counts_every_line(shape, npml, esize):
    assert bench.cpml_bytes_per_step(shape, npml, esize) == pytest.approx(
        _enumerate_cpml(shape, npml, esize), rel=1e-12)


def test_cpml_gradient_bytes_per_step_counts_every_line():
    """72 B per point (forward 16, recompute with D 20, adjoint 36) plus per
    line: the forward's layer pass (16 B at segment points and slab cells),
    the recompute's (the same + D read and written at the segment points)
    and the adjoint's (p^{k+1}, C, p^k read and written at the segment
    points; nu, mu read and written at the slab cells)."""
    shape, npml = (40, 36, 44), 8
    nx, ny, nz = shape
    w = npml + 4
    total = 72 * nx * ny * nz
    for n, nlines in ((nx, ny * nz), (ny, nx * nz), (nz, nx * ny)):
        seg = sum(1 for i in range(n) if i < w or i >= n - w)
        slab = sum(1 for i in range(n) if i < npml or i >= n - npml)
        fwd = 16 * seg + 16 * slab
        rec = fwd + 8 * seg
        adj = 16 * seg + 16 * slab
        total += nlines * (fwd + rec + adj)
    assert bench.cpml_gradient_bytes_per_step(shape, npml) == pytest.approx(total, rel=1e-12)


def test_traffic_is_reported_only_for_the_current_kernel_sources(tmp_path):
    good = tmp_path / "good.txt"
    good.write_text("# comment: a line with a colon\nkernel_source_sha256_16: %s\n"
                    "dram_bytes_per_launch[wl]: 1.5e+09\n" % bench.kernel_hash())
    stale = tmp_path / "stale.txt"
    stale.write_text("kernel_source_sha256_16: 0000000000000000\n"
                     "dram_bytes_per_launch[wl]: 1.5e+09\n")
    assert bench.read_traffic("wl", str(good)) == 1.5e9
    assert bench.read_traffic("other", str(good)) is None
    assert bench.read_traffic("wl", str(stale)) is None
    assert bench.read_traffic("wl", str(tmp_path / "missing.txt")) is None
