"""Host logic of the z-layer plan (no GPU): a host program compiled with nvcc
from the library's own source calls plan_layers and layer_makespan.

A sweep launch gives each CTA an xy tile and a range of z planes (a layer).
The planner splits nz into at most 16 layers by a makespan model in which a
CTA runs planes + 4 stages (8 for the 16-bit sweeps) and every resident CTA advances one stage per
1 + C / slots time units while C CTAs are resident (latency bound alone,
sharing HBM bandwidth when many run). The fixed plans below are the ones
measured fastest on GB300 among the plans timed for each grid (FP32, 32 x 16
tiles, 4 CTAs per SM on 152 SMs).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SLOTS = 152 * 4


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("plan") / "layer_plan")
    subprocess.run([nvcc, "-std=c++17", "-O2", os.path.join(ROOT, "tests", "host", "layer_plan.cu"),
                    "-o", exe], check=True, capture_output=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout.split("\n")
        return [l for l in out if l.strip()]
    return run


def tiles(nx, ny):
    return -(-nx // 32) * -(-ny // 16)


def plan_of(planner, nx, ny, nz, slots=SLOTS):
    line = planner(["%d %d %d" % (nz, tiles(nx, ny), slots)])[0].split()
    return float(line[0]), [int(v) for v in line[1:]]


@pytest.mark.parametrize("dims,expected", [
    ((1024, 1024, 512), [272, 216, 24]),
    ((512, 512, 512), [448, 64]),
    ((448, 448, 448), [150, 150, 148]),
    ((320, 320, 320), [107, 107, 106]),
    ((256, 256, 256), [64] * 4),
    ((192, 192, 192), [24] * 8),
    ((160, 480, 288), [72] * 4),
    ((128, 128, 128), [8] * 16),
])
def test_plans_measured_fastest(planner, dims, expected):
    assert plan_of(planner, *dims)[1] == expected


@pytest.mark.parametrize("dims,expected", [
    ((1024, 1024, 512), [448, 64]),
    ((512, 512, 512), [448, 64]),
])
def test_plans_16bit(planner, dims, expected):
    # the 16-bit sweeps (64 x 8 tiles, same tile counts) plan with preroll 8
    nx, ny, nz = dims
    nt = -(-nx // 64) * -(-ny // 8)
    line = planner(["%d %d %d 8" % (nz, nt, SLOTS)])[0].split()
    assert [int(v) for v in line[1:]] == expected


@pytest.mark.parametrize("nz", [1, 2, 7, 16, 17, 100, 255, 1040, 4096])
@pytest.mark.parametrize("ntiles", [1, 5, 128, 2048, 8192])
def test_plans_cover_the_grid(planner, nz, ntiles):
    line = planner(["%d %d %d" % (nz, ntiles, SLOTS)])[0].split()
    ch = [int(v) for v in line[1:]]
    assert sum(ch) == nz and 1 <= len(ch) <= 16 and min(ch) >= 1


def test_single_cta_and_more_slots(planner):
    # one CTA alone: (planes + 4) stages at 1 + 1/slots each
    for k in (1, 8, 100):
        v = float(planner(["makespan 1 %d %d" % (SLOTS, k)])[0])
        assert abs(v - (k + 4) * (1 + 1 / SLOTS)) < 1e-9
    # the same plan never takes longer with more resident places
    plan = "272 216 24"
    vals = [float(planner(["makespan 2048 %d %s" % (s, plan)])[0]) for s in (152, 304, 608, 1216)]
    assert all(a >= b - 1e-9 for a, b in zip(vals, vals[1:]))
    # and a plan of n equal CTAs that all fit runs as long as one CTA at
    # concurrency n
    v = float(planner(["makespan 100 %d 60" % SLOTS])[0])
    assert abs(v - 64 * (1 + 100 / SLOTS)) < 1e-9
