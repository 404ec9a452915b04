"""Pins of the oracle's random streams (Philox4x32-10 and its variate maps)."""
import fractions
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _torch_ref_binary(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    torch_ext = pytest.importorskip("torch.utils.cpp_extension")
    out = str(tmp_path_factory.mktemp("philox") / "philox_torch_ref")
    inc = []
    for p in torch_ext.include_paths():
        inc += ["-I", p]
    subprocess.run(["g++", "-O1", "-std=c++17", *inc, os.path.join(HERE, "philox_torch_ref.cpp"),
                    "-o", out], check=True)
    return out


def test_philox_matches_aten_engine(orc, tmp_path_factory):
    """Counter blocks agree with PyTorch's ATen philox_engine on random keys/counters."""
    exe = _torch_ref_binary(tmp_path_factory)
    g = np.random.default_rng(1234)
    seeds = [0, 1, 0xFFFFFFFFFFFFFFFF] + [int(x) for x in g.integers(0, 2**63, 60)]
    subs = [0, 0xFFFFFFFFFFFFFFFF] + [int(x) for x in g.integers(0, 2**63, 61)]
    offs = [0, 0xFFFFFFFFFFFFFFFF] + [int(x) for x in g.integers(0, 2**63, 61)]
    lines = "".join(f"{s} {b} {o}\n" for s, b, o in zip(seeds, subs, offs))
    res = subprocess.run([exe], input=lines, capture_output=True, text=True, check=True)
    ref = [[int(w, 16) for w in ln.split()] for ln in res.stdout.strip().splitlines()]
    for (s, b, o), r in zip(zip(seeds, subs, offs), ref):
        ctr = [o & 0xFFFFFFFF, o >> 32, b & 0xFFFFFFFF, b >> 32]
        got = orc.philox(ctr, orc.seed_key(s))
        assert list(map(int, got)) == r, (s, b, o)


def test_philox_words_uniform(orc):
    """Chi-square of 2^20 words over 256 bins of the top byte, and bit balance."""
    n = 1 << 18
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 1] = 7
    ctr[:, 3] = (3 << 24)
    w = orc.philox(ctr, orc.seed_key(99)).ravel()
    counts = np.bincount(w >> 24, minlength=256)
    exp = w.size / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # 255 dof: mean 255, sd ~22.6; 6 sd band
    assert 120 < chi2 < 400, chi2
    bits = np.unpackbits(w.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 1e-3


def test_philox_counter_sensitivity(orc):
    """Every counter word and both key words change the block (no ignored input)."""
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(orc.philox(c, [5, 6]), base)
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert not np.array_equal(orc.philox([1, 2, 3, 4], k), base)


def test_uniform_f32_is_one_fma_rounding(orc):
    """U(a,b) equals the exactly rounded (b-a)*u + a computed in rationals."""
    g = np.random.default_rng(5)
    for a, b in [(-0.05, 0.05), (-3.0, 3.0), (-0.5, 0.5), (-0.2041241452, 0.2041241452)]:
        a32, b32 = np.float32(a), np.float32(b)
        d = np.float32(b32 - a32)
        for w in g.integers(0, 2**32, 2000):
            u = fractions.Fraction(int(w) >> 8, 1 << 24)
            exact = fractions.Fraction(float(d)) * u + fractions.Fraction(float(a32))
            ref = np.float32(float(exact))  # float() of a Fraction rounds correctly to FP64
            # FP64 -> FP32 double rounding is impossible here: exact has <= 53 bits
            assert fractions.Fraction(float(exact)) == exact
            got = orc.uniform_f32(int(w), a32, b32)
            assert got == ref
            assert a32 <= got <= b32


def test_u01_and_bounded(orc):
    assert orc.u01(0) == 0.0
    assert orc.u01(0xFFFFFFFF) == (2**24 - 1) / 2**24
    assert orc.u01(0x00000100) == 2.0**-24
    for n in [1, 7, 249, 990001]:
        assert orc.bounded(0, n) == 0
        assert orc.bounded(0xFFFFFFFF, n) == n - 1
    # multiply-shift is exact integer floor(w*n/2^32)
    g = np.random.default_rng(3)
    for w in g.integers(0, 2**32, 500):
        assert orc.bounded(int(w), 249) == (int(w) * 249) >> 32


def test_box_muller_moments(orc):
    """Normals from Box-Muller: mean 0, var 1, and the cos/sin pair uncorrelated."""
    n = 1 << 16
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    w = orc.philox(ctr, orc.seed_key(11))
    zs = np.array([orc.box_muller(int(a), int(b)) for a, b in w[:, :2]])
    assert abs(zs.mean()) < 0.02
    assert abs(zs.var() - 1.0) < 0.03
    assert abs(np.corrcoef(zs[:, 0], zs[:, 1])[0, 1]) < 0.02
    scipy_stats = pytest.importorskip("scipy.stats")
    assert scipy_stats.kstest(zs[:, 0], "norm").pvalue > 1e-4
    # extreme words: u1 = 2^-24 gives the largest radius, u1 = 1 gives zero
    zc, _ = orc.box_muller(0, 0)
    assert zc == pytest.approx(np.sqrt(-2 * np.log(2.0**-24)))
    zc, zsn = orc.box_muller(0xFFFFFFFF, 0)
    assert zc == 0.0 and zsn == 0.0


def test_round_bf16_matches_torch(orc):
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(8)
    x = np.concatenate([g.standard_normal(4000), g.uniform(-1e4, 1e4, 1000),
                        [0.0, 1.0, -1.0, 1.00390625, 1.005859375]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([orc.round_bf16(v) for v in x], np.float32)
    assert np.array_equal(got, ref)
