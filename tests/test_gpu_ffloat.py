"""Float-float arithmetic of the FP32 inner loops (ffloat.cuh), run on the GPU
by a small harness and checked against exact rational arithmetic.

The FP32 inner CG loops keep their reductions and scalar updates in pairs of
FP32 numbers instead of FP64 (GB300's FP64 rate would put microseconds of FP64
on every iteration).  The pairs must (1) meet the published error bounds of
the double-word algorithms they follow (Joldes, Muller and Popescu 2017:
sum <= 3u^2, sum with one FP32 number <= 2u^2, u = 2^-24; the product and the
quotient are held to 8u^2 here), (2) give the same bits for a + b and b + a
(the butterfly reductions rely on it: every lane, and every CTA, must end
with the same state), (3) sum per-CTA pairs to within n * 3u^2 of the exact
sum, and (4) take the same decisions as the FP64 scalar update with alpha and
beta equal to 1e-12.
"""
import os
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "ff_harness.cu")
U = Fraction(1, 2**24)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    from paper_1908_03301_gb300 import build as b

    exe = str(tmp_path_factory.mktemp("ff") / "ff_harness")
    nvcc = b.NVCC if os.path.exists(b.NVCC) else "nvcc"
    subprocess.run([nvcc, *b.ARCH, "-O3", "-std=c++17", SRC, "-o", exe], check=True, capture_output=True)
    return exe


def pairs_of(d):
    """Normalised pairs (hi, lo) of float64 values."""
    h = d.astype(np.float32)
    l = (d - h.astype(np.float64)).astype(np.float32)
    return h, l


def exact(h, l):
    return Fraction(float(h)) + Fraction(float(l))


def run(exe, tmp, ops, slots, fin_v, fin_i):
    inp, out = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
    with open(inp, "wb") as f:
        f.write(struct.pack("<3i", len(ops), len(slots), len(fin_v)))
        f.write(np.ascontiguousarray(ops, dtype=np.float32).tobytes())
        f.write(np.ascontiguousarray(slots, dtype=np.float32).tobytes())
        rec = np.zeros(len(fin_v), dtype=[("v", "<f8", 9), ("i", "<i8", 5)])
        rec["v"], rec["i"] = fin_v, fin_i
        f.write(rec.tobytes())
    subprocess.run([exe, inp, out], check=True, capture_output=True, timeout=120)
    raw = open(out, "rb").read()
    n, m, k = len(ops), len(slots), len(fin_v)
    o = np.frombuffer(raw, dtype=np.float32, count=n * 14).reshape(n, 7, 2)
    off = n * 14 * 4
    s = np.frombuffer(raw, dtype=np.float32, count=2 * 32 * 8, offset=off).reshape(2, 32, 4, 2)
    off += 2 * 32 * 8 * 4
    fo = np.dtype([("d", "<f8", 5), ("i", "<i8", 2)])
    r_ff = np.frombuffer(raw, dtype=fo, count=k, offset=off)
    r_d = np.frombuffer(raw, dtype=fo, count=k, offset=off + k * fo.itemsize)
    return o, s, r_ff, r_d


def random_values(gen, n, lo_exp=-20, hi_exp=20):
    mag = np.ldexp(gen.uniform(1.0, 2.0, n), gen.integers(lo_exp, hi_exp, n))
    return mag * gen.choice([-1.0, 1.0], n)


def test_pair_operations_meet_error_bounds(harness, tmp_path):
    gen = np.random.default_rng(20240611)
    n = 3000
    a = random_values(gen, n)
    b = random_values(gen, n)
    # cancellation cases: b close to -a and to a
    b[:500] = -a[:500] * (1.0 + gen.uniform(-1e-6, 1e-6, 500))
    b[500:1000] = a[500:1000] * (1.0 + gen.uniform(-1e-9, 1e-9, 500))
    ah, al = pairs_of(a)
    bh, bl = pairs_of(b)
    ops = np.stack([ah, al, bh, bl], axis=1)
    slots = np.zeros((1, 8), np.float32)
    fin_v = np.ones((1, 9))
    fin_i = np.array([[0, 0, 0, 10, 10]])
    o, _, _, _ = run(harness, str(tmp_path), ops, slots, fin_v, fin_i)
    bound = {0: 3 * U * U, 1: 3 * U * U, 2: 8 * U * U, 3: 8 * U * U, 4: 2 * U * U}
    worst = {k: Fraction(0) for k in bound}
    for i in range(n):
        x, y = exact(ah[i], al[i]), exact(bh[i], bl[i])
        want = {0: x + y, 1: x - y, 2: x * y, 3: x / y, 4: x + Fraction(float(bh[i]))}
        for k, w in want.items():
            got = exact(o[i, k, 0], o[i, k, 1])
            if w == 0:
                assert got == 0, (i, k)
                continue
            err = abs(got - w) / abs(w)
            worst[k] = max(worst[k], err)
            assert err <= bound[k], (i, k, float(err / (U * U)))
            # the result is a normalised pair: |lo| <= ulp(hi) / 2
            h, l = float(o[i, k, 0]), float(o[i, k, 1])
            assert abs(l) <= np.spacing(np.float32(abs(h))) / 2, (i, k, h, l)
        # a + b and b + a: the same bits
        assert o[i, 5, 0] == o[i, 0, 0] and o[i, 5, 1] == o[i, 0, 1], i
        # b * a: same bound as a * b
        got = exact(o[i, 6, 0], o[i, 6, 1])
        assert abs(got - want[2]) <= bound[2] * abs(want[2]), i
    # the check has teeth: FP32 alone would be off by up to u / 2
    assert all(float(w) < 2.0**-44 for w in worst.values())


@pytest.mark.parametrize("n", [1, 31, 33, 152, 304, 1000])
def test_warp_sum_of_slots(harness, tmp_path, n):
    gen = np.random.default_rng(5000 + n)
    vals = np.stack([random_values(gen, n, -8, 8) for _ in range(4)], axis=1)
    vals[:, 1] = np.abs(vals[:, 1])  # one all-positive column
    h, l = pairs_of(vals)
    slots = np.concatenate([h, l], axis=1)  # hi[4], lo[4] per slot
    ops = np.zeros((1, 4), np.float32)
    ops[0] = [1, 0, 1, 0]
    _, s, _, _ = run(harness, str(tmp_path), ops, slots, np.ones((1, 9)), np.array([[0, 0, 0, 10, 10]]))
    for depth in range(2):  # four, then five slots per lane in flight
        sd = s[depth]
        # every lane holds the same bits
        assert np.array_equal(sd, np.broadcast_to(sd[0], sd.shape))
        for k in range(4):
            terms = [exact(h[i, k], l[i, k]) for i in range(n)]
            want = sum(terms, Fraction(0))
            scale = sum((abs(t) for t in terms), Fraction(0))
            got = exact(sd[0, k, 0], sd[0, k, 1])
            assert abs(got - want) <= max(n, 2) * 3 * U * U * scale, (depth, k, float(abs(got - want) / scale))


def test_scalar_update_matches_fp64(harness, tmp_path):
    gen = np.random.default_rng(77)
    n = 4000
    rr = np.ldexp(gen.uniform(1, 2, n), gen.integers(-40, 40, n))
    pq = rr * gen.uniform(0.05, 20.0, n)
    a = rr / pq
    # <r,q> and <q,q> from a plausible ||r - a q||^2 = rr * beta, beta in (0, 1.2)
    qq = pq * gen.uniform(0.5, 4.0, n) / 1.0
    beta = gen.uniform(1e-4, 1.2, n)
    rq = (rr + a * a * qq - beta * rr) / (2.0 * a)
    tol2 = np.ldexp(1.0, gen.integers(-60, -2, n))
    rho0 = rr * np.ldexp(1.0, gen.integers(0, 30, n))
    delta2 = np.where(gen.random(n) < 0.5, 1e-6, 0.0)
    maxrr = rr * gen.uniform(0.5, 1e7, n)
    best = rr * gen.uniform(0.5, 8.0, n)
    reliable = (gen.random(n) < 0.5).astype(np.int64)
    it = gen.integers(0, 1000, n)
    best_iter = it - gen.integers(0, 400, n)
    max_iter = it + gen.integers(0, 3, n)
    stag = np.full(n, 300)
    # special cases: zero residual, non-positive <p,q>, cancellation to 0
    rr[:20] = 0.0
    best[:20] = 1.0
    pq[20:40] = -pq[20:40]
    rq[40:60] = (rr[40:60] + a[40:60] ** 2 * qq[40:60]) / (2 * a[40:60])
    v = np.stack([pq, rq, qq, rr, tol2, rho0, delta2, maxrr, best], axis=1)
    ii = np.stack([reliable, it, best_iter, max_iter, stag], axis=1)
    # inputs exactly representable as pairs, so both updates see the same sums
    for j in range(4):
        h, l = pairs_of(v[:, j])
        v[:, j] = h.astype(np.float64) + l.astype(np.float64)
    _, _, r_ff, r_d = run(harness, str(tmp_path), np.zeros((1, 4), np.float32), np.zeros((1, 8), np.float32), v, ii)
    # skip near-ties of a threshold test (decided by the last bits), in the
    # order the update takes its decisions
    pq_, rq_, qq_, rr_ = v[:, 0], v[:, 1], v[:, 2], v[:, 3]
    thr = v[:, 4] * v[:, 5]

    def near(x, y):
        return np.abs(x - y) <= 1e-6 * np.maximum(np.abs(x), np.abs(y))

    live = (rr_ > 0) & (pq_ > 0)
    a2 = np.where(live, rr_ / np.where(pq_ != 0, pq_, 1.0), 0.0)
    terms = rr_ + np.abs(2.0 * a2 * rq_) + a2 * a2 * qq_
    rn1 = rr_ - 2.0 * a2 * rq_ + a2 * a2 * qq_
    mx = np.maximum(v[:, 7], rr_)
    tie = (rr_ > 0) & (ii[:, 0] == 0) & near(rr_, thr)
    tie |= live & (near(rn1, thr) | near(rn1, v[:, 6] * mx) | near(rr_, 0.25 * v[:, 8]))
    tie |= live & (np.abs(rn1) <= 1e-6 * terms)  # cancellation to ~0 decided by rounding
    keep = ~tie
    assert keep.sum() > 0.9 * n
    np.testing.assert_array_equal(r_ff["i"][keep], r_d["i"][keep])
    # alpha, rho, best, maxrr to 1e-12; beta to 1e-12 of the terms it cancels
    for j in (0, 2, 3, 4):
        np.testing.assert_allclose(r_ff["d"][keep, j], r_d["d"][keep, j], rtol=1e-12, atol=0, err_msg=f"field {j}")
    db = np.abs(r_ff["d"][keep, 1] - r_d["d"][keep, 1])
    scale = np.where(rr_[keep] > 0, terms[keep] / np.where(rr_[keep] > 0, rr_[keep], 1.0), 1.0)
    assert np.all(db <= 1e-12 * scale), float(np.max(db / scale))
    codes = set(r_d["i"][keep, 0].tolist())
    assert {0, 1, 4, 6} <= codes, codes  # running, converged, breakdown, refinement due
