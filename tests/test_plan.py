"""Host-side work planning of the sweep kernel (no GPU).

The planner cuts networks into segments (column block x row band x march
range) and deals them to CTAs.  A plan must cover every lattice node of every
network exactly once, give each network's segments distinct partial-sum
slots, keep column blocks 16-byte aligned and within the kernel's patch
limits, and balance the CTAs: a sweep launch lasts as long as its slowest CTA.
The harness links the library's own planner objects and prints the plan.
"""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS_SRC = os.path.join(ROOT, "tests", "native", "plan_harness.cu")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    from paper_1908_03301_gb300 import build as b

    b.build()
    objdir = os.path.join(b.OUT, "obj")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_harness")
    nvcc = b.NVCC if os.path.exists(b.NVCC) else "nvcc"
    subprocess.run([nvcc, *b.ARCH, "-std=c++17", "-I", os.path.join(ROOT, "include"), HARNESS_SRC,
                    os.path.join(objdir, "plan.cu.o"), os.path.join(objdir, "sweep.cu.o"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def run_plan(exe, ndim, f32, nsm, shape, dims_list):
    args = [exe, str(ndim), str(f32), str(nsm), *[str(v) for v in shape]]
    for d in dims_list:
        d = list(d) + [1] * (3 - len(d))
        args += [str(v) for v in d]
    out = subprocess.run(args, check=True, capture_output=True, text=True).stdout.split("\n")
    if out[0] == "invalid":
        return None
    grid = int(out[0].split()[1])
    segs, nseg, cap = [], {}, None
    for line in out[1:]:
        if not line:
            continue
        f = line.split()
        if f[0] == "nseg":
            nseg[int(f[1])] = int(f[2])
        elif f[0] == "cap":
            cap, wmax = int(f[1]), int(f[3])
        else:
            segs.append(tuple(int(v) for v in f))
    return grid, segs, nseg, cap, wmax


def step_cost(ndim, f32, w, h, px, x0):
    """The planner's cost of one march step: its nodes plus 100 node-equivalents
    per bulk copy.  2D stages hold several rows (one copy per array over whole
    rows, one per row otherwise): a slot holds 2080 floats / 1040 doubles.  A
    2D row costs at least 270 node-equivalents (the consumers' fixed time per
    row)."""
    full = x0 == 0 and w == px
    if ndim == 2:
        cap, V = (2080, 4) if f32 else (1040, 2)
        R = (cap - 2 * V) // px if full else cap // (w + 2 * V)
        R = max(1, min(16, R))
        copies = 6 / R if full else 6
        return w * h + max(100 * copies, 270)
    copies = 7 if full else 3 * (h + 2) + 4 * h + 1
    return w * h + 100 * copies


def check_plan(plan, ndim, dims_list, f32=1):
    grid, segs, nseg, cap, wmax = plan
    cover = []
    for d in dims_list:
        nx, ny = d[0], d[1]
        nz = d[2] if ndim == 3 else 1
        px = (nx + 3) // 4 * 4
        cover.append(np.zeros((nz, ny, px), np.int32))
    slots = [set() for _ in dims_list]
    load = np.zeros(grid)
    for cta, inst, x0, w, y0, h, m0, m1, slot in segs:
        assert 0 <= cta < grid
        assert x0 % 4 == 0 and w % 4 == 0 and 0 < w <= wmax
        assert 0 <= m0 < m1
        if ndim == 3:
            assert w * h <= cap and 1 <= h <= 32
            cover[inst][m0:m1, y0:y0 + h, x0:x0 + w] += 1
        else:
            assert h == 1 and y0 == 0
            cover[inst][0, m0:m1, x0:x0 + w] += 1
        assert slot not in slots[inst]
        slots[inst].add(slot)
        load[cta] += step_cost(ndim, f32, w, h, (dims_list[inst][0] + 3) // 4 * 4, x0) * (m1 - m0 + 2)
    for k, c in enumerate(cover):
        assert (c == 1).all(), f"network {k}: nodes covered {c.min()}..{c.max()} times"
        assert slots[k] == set(range(nseg[k]))
    busy = load[load > 0]
    # slowest CTA against a perfect split of the same work over all CTAs
    return load.max() / (load.sum() / grid), len(busy)


@pytest.mark.parametrize("ndim,dims_list", [
    (3, [(192, 192, 192)]),
    (3, [(256, 256, 256)]),
    (3, [(37, 29, 23)]),
    (2, [(4096, 4096)]),
    (2, [(3000, 17)]),
])
def test_single_network_plans_cover_and_balance(harness, ndim, dims_list):
    plan = run_plan(harness, ndim, 1, 152, (0, 0, 1), dims_list)
    imb, busy = check_plan(plan, ndim, dims_list)
    big = np.prod(dims_list[0]) > 10**6
    if big:
        # equal pieces: the slowest CTA within a few % of a perfect split
        assert imb <= 1.06, (imb, busy)


def test_batch_plan_covers_and_balances(harness):
    gen = np.random.default_rng(1)
    dims_list = [(int(s), int(s)) for s in gen.integers(64, 1025, size=120)]
    for shape in [(0, 0, 1), (0, 0, 2), (512, 0, 4), (256, 0, 1)]:
        plan = run_plan(harness, 2, 1, 152, shape, dims_list)
        imb, busy = check_plan(plan, 2, dims_list)
        assert imb <= 1.06, (shape, imb)


def test_3d_shapes_and_fp64(harness):
    dims_list = [(41, 27, 19), (70, 64, 66), (16, 16, 16)]
    for f32, shapes in [(1, [(256, 4, 1), (128, 8, 2), (64, 16, 4), (32, 32, 1), (16, 0, 3)]),
                        (0, [(128, 4, 1), (64, 8, 2), (32, 16, 1), (0, 0, 2)])]:
        for shape in shapes:
            plan = run_plan(harness, 3, f32, 152, shape, dims_list)
            assert plan is not None, shape
            check_plan(plan, 3, dims_list, f32)


def test_invalid_shapes_are_rejected(harness):
    assert run_plan(harness, 3, 1, 152, (256, 8, 1), [(20, 20, 20)]) is None  # 2048 > 1024 per step
    assert run_plan(harness, 2, 1, 152, (6, 0, 1), [(20, 20)]) is None        # not a multiple of 4
    assert run_plan(harness, 3, 0, 152, (256, 4, 1), [(20, 20, 20)]) is None  # FP64 max width 128
    assert run_plan(harness, 2, 1, 152, (0, 0, 0), [(20, 20)]) is None


def test_tiny_networks_and_few_sms(harness):
    dims_list = [(4, 3), (5, 9), (8, 8), (12, 4)]
    plan = run_plan(harness, 2, 1, 3, (0, 0, 1), dims_list)
    check_plan(plan, 2, dims_list)
    plan = run_plan(harness, 3, 1, 7, (0, 0, 2), [(3, 4, 5), (9, 2, 3)])
    check_plan(plan, 3, [(3, 4, 5), (9, 2, 3)])
