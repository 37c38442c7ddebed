"""The seeded input generators against their stated recipe (CPU only).

Every workload is drawn from one counter-based generator (splitmix64) and
shaped into the benchmark's distributions.  These tests pin the generator
to the published splitmix64 outputs and check each distribution for the
property its recipe promises: the order of sorted / reverse inputs, at most
16 distinct values for dup16, the Zipf(1) head frequencies, the normal
moments and the special-value rate of the pairs, the log-uniform segment
lengths.  None of it involves the sort."""
import math

import numpy as np
import pytest

from paper_2409_03970_gb300 import inputs

M64 = (1 << 64) - 1


def mix64_int(z: int) -> int:
    """splitmix64's finaliser on a Python int (the definition, mod 2^64)."""
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & M64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_mix64_gives_the_published_splitmix64_outputs():
    """SplitMix64 seeded with 0 (Steele, Lea and Flood, OOPSLA 2014; the
    reference generator adds 0x9E3779B97F4A7C15 to the state before each
    output) starts 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F."""
    states = np.array([(k * 0x9E3779B97F4A7C15) & M64 for k in (1, 2, 3)], dtype=np.uint64)
    got = [int(v) for v in inputs.mix64(states)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("seed,stream", [(0, 0), (7, 3), (123456, 7)])
def test_counter_draws_follow_the_stated_formula(seed, stream):
    base = mix64_int((seed * 65536 + stream + 1) & M64)
    want = [mix64_int((base + (i + 1) * 0x9E3779B97F4A7C15) & M64) for i in range(5, 12)]
    assert [int(v) for v in inputs.counter_u64(seed, stream, 5, 12)] == want
    assert [int(v) for v in inputs.counter_u32(seed, stream, 5, 12)] == [w >> 32 for w in want]


def test_draws_are_deterministic_and_chunk_independent():
    a = inputs.keys(inputs.CHUNK + 1000, "u32", "uniform", seed=5)
    assert np.array_equal(a, inputs.keys(inputs.CHUNK + 1000, "u32", "uniform", seed=5))
    assert np.array_equal(a[:1000], inputs.keys(1000, "u32", "uniform", seed=5))
    assert not np.array_equal(a[:1000], inputs.keys(1000, "u32", "uniform", seed=6))


def test_uniform_covers_each_dtype_range():
    n = 1 << 18
    u = inputs.keys(n, "u32", "uniform", seed=1)
    assert abs(u.astype(np.float64).mean() / 2**32 - 0.5) < 0.01
    top = np.bincount((u >> 28).astype(np.int64), minlength=16)
    assert top.min() > 0.9 * n / 16 and top.max() < 1.1 * n / 16
    i = inputs.as_dtype(inputs.keys(n, "i32", "uniform", seed=1), "i32")
    assert 0.45 < (i < 0).mean() < 0.55
    f = inputs.as_dtype(inputs.keys(n, "f32", "uniform", seed=1), "f32")
    assert np.isfinite(f).all() and f.min() >= -1.0 and f.max() < 1.0
    assert abs(f.mean()) < 0.01


@pytest.mark.parametrize("dt", inputs.KEY_DTYPES)
def test_sorted_and_reverse_are_ordered_in_the_dtype(dt):
    n = 100_003
    s = inputs.as_dtype(inputs.keys(n, dt, "sorted", seed=2), dt)
    r = inputs.as_dtype(inputs.keys(n, dt, "reverse", seed=2), dt)
    assert np.all(s[1:] >= s[:-1])
    assert np.all(r[1:] <= r[:-1])
    assert len(np.unique(s)) > 0.9 * n          # spread over the range, not clumped


@pytest.mark.parametrize("dt", inputs.KEY_DTYPES)
def test_dup16_has_at_most_16_values_all_used(dt):
    x = inputs.keys(50_000, dt, "dup16", seed=3)
    vals, counts = np.unique(x, return_counts=True)
    assert len(vals) <= 16 and counts.min() > 50_000 / 16 * 0.8


def test_zipf_head_frequencies_follow_one_over_rank():
    """Zipf(s=1) over R = 2^20 ranks: rank r has probability 1 / (r H_R),
    with H_R the R-th harmonic number."""
    n, R = 1 << 20, 1 << 20
    H = math.fsum(1.0 / r for r in range(1, R + 1))
    x = inputs.keys(n, "u32", "zipf", seed=4)
    _, counts = np.unique(x, return_counts=True)
    top = np.sort(counts)[::-1][:4] / n
    for r, p in enumerate(top, start=1):
        assert abs(p - 1.0 / (r * H)) < 0.15 / (r * H)


def test_normal_pairs_moments_specials_and_payload():
    n = 1 << 20
    k, v = inputs.normal_pairs(n, seed=5)
    assert np.array_equal(v, np.arange(n, dtype=np.uint32))
    special = np.isin(k, inputs.SPECIALS_F32)
    assert 0.0007 < special.mean() < 0.0013               # about 1 per mille
    z = k[~special].view(np.float32).astype(np.float64)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert abs((np.abs(z) < 1.0).mean() - 0.6827) < 0.005   # the normal's one-sigma mass
    assert len(np.unique(k[special])) >= 5                   # several of the seven specials


def test_segment_offsets_are_log_uniform_csr():
    nseg = 100_000
    off = inputs.segment_offsets(nseg, seed=0)
    lens = np.diff(off)
    assert off[0] == 0 and np.all(lens >= 1) and lens.max() <= 65536
    # the benchmark's batch: 588,066,542 keys
    assert int(off[-1]) == 588_066_542
    # log2 of the length is uniform on [0, 16): each unit octave holds 1/16
    octave = np.floor(np.log2(lens)).astype(np.int64)
    frac = np.bincount(octave, minlength=17)[:16] / nseg
    assert np.all(np.abs(frac - 1 / 16) < 0.005)
    # mean length: integral of 2^(16u) du = (2^16 - 1) / (16 ln 2), less the floor
    assert abs(lens.mean() - (65535 / (16 * math.log(2)) - 0.5)) < 0.02 * lens.mean()


@pytest.mark.parametrize("dt", inputs.KEY64_DTYPES)
def test_keys64_orders_and_values(dt):
    n = 50_001
    s = inputs.keys64(n, dt, "sorted", seed=6)
    view = {"u64": np.uint64, "i64": np.int64, "f64": np.float64}[dt]
    sv = s.view(view)
    assert np.all(sv[1:] >= sv[:-1])
    assert len(np.unique(inputs.keys64(n, dt, "dup16", seed=6))) <= 16
    if dt == "f64":
        u = inputs.keys64(n, dt, "uniform", seed=6).view(np.float64)
        assert np.isfinite(u).all() and u.min() >= -1.0 and u.max() < 1.0
