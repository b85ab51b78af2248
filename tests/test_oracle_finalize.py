"""Pins for the oracle's finalizer: variance under the posterior and PAC noise.

Sec. 2 "PAC Privacy": release f(S) + N(0, Var_{P}[f] / (2B)) and, for a
sequence of releases, take the variance under the current posterior P and
update P by Bayes' rule after each release.  Sec. 4.1 gives the four steps of
the noise function; Sec. 2 adds the factor 2 of pac_noised_count; Sec. 3.2
adds the NULL mechanism; Sec. 5 the diversity check.  The pins check these
against library routines (numpy's population variance, scipy's normal pdf)
and against statistics that hold for any correct implementation.
"""
import numpy as np
import pytest
from scipy import stats

FULL = np.uint64(0xFFFFFFFFFFFFFFFF)


def _z(orc, seed, cell):
    return orc.lib().orc_box_muller(orc.rng_u64(seed, 2, 2 * cell), orc.rng_u64(seed, 2, 2 * cell + 1))


def test_release_scale(orc):
    assert orc.release_scale(orc.COUNT) == 2.0
    assert orc.release_scale(orc.SUM) == 2.0
    for k in (orc.AVG, orc.MIN, orc.MAX):
        assert orc.release_scale(k) == 1.0


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_huge_budget_releases_scaled_secret_world(orc, kind):
    # B -> infinity: no noise, the release is scale * y[j*]  (Sec. 2: count[j*]*2)
    rng = np.random.default_rng(kind)
    for seed in range(20):
        y = rng.integers(0, 1000, size=(1, 1, 64)).astype(np.float64)
        out = orc.finalize(y, [orc.release_scale(kind)], np.array([500], np.uint64),
                           np.array([FULL]), seed, 1e300)
        js = out["jstar"]
        assert out["noised"][0] == pytest.approx(orc.release_scale(kind) * y[0, 0, js], rel=1e-12)


def test_uniform_posterior_noise_scale(orc):
    """Independent mode (P uniform per cell): (release - y[j*]) / sqrt(var/(2B))
    is standard normal, var = numpy's population variance of the scaled y."""
    rng = np.random.default_rng(5)
    G, B = 4000, 1.0 / 128
    y = rng.lognormal(5, 1, size=(G, 1, 64))
    res = []
    for seed in (1, 2):
        out = orc.finalize(y, [2.0], np.full(G, 1000, np.uint64), np.full(G, FULL), seed, B,
                           orc.INDEPENDENT)
        js = out["jstar"]
        sy = 2.0 * y[:, 0, :]
        sd = np.sqrt(np.var(sy, axis=1) / (2 * B))
        res.append((out["noised"] - sy[:, js]) / sd)
    r = np.concatenate(res)
    assert stats.kstest(r, "norm").pvalue > 1e-3
    # and it is exactly the seeded draw
    out = orc.finalize(y[:3], [2.0], np.full(3, 1000, np.uint64), np.full(3, FULL), 9, B,
                       orc.INDEPENDENT)
    sy = 2.0 * y[:3, 0, :]
    for c in range(3):
        expect = sy[c, out["jstar"]] + np.sqrt(np.var(sy[c]) / (2 * B)) * _z(orc, 9, c)
        assert out["noised"][c] == pytest.approx(expect, rel=1e-12)


def test_bayes_update_matches_normal_likelihood(orc):
    """Two adaptive releases: the second variance is taken under the
    posterior after the first, P1 ~ P0 * N(y1~; y1_j, Delta1) (scipy pdf)."""
    rng = np.random.default_rng(8)
    B = 0.5
    y = rng.normal(100, 10, size=(2, 1, 64))
    seed = 77
    out = orc.finalize(y, [1.0], np.full(2, 100, np.uint64), np.full(2, FULL), seed, B)
    js = out["jstar"]
    p0 = np.full(64, 1 / 64)
    d1 = np.var(y[0, 0]) / (2 * B)
    yt1 = y[0, 0, js] + np.sqrt(d1) * _z(orc, seed, 0)
    assert out["noised"][0] == pytest.approx(yt1, rel=1e-12)
    p1 = p0 * stats.norm.pdf(yt1, loc=y[0, 0], scale=np.sqrt(d1))
    p1 /= p1.sum()
    mu2 = np.sum(p1 * y[1, 0])
    d2 = np.sum(p1 * (y[1, 0] - mu2) ** 2) / (2 * B)
    yt2 = y[1, 0, js] + np.sqrt(d2) * _z(orc, seed, 1)
    assert out["noised"][1] == pytest.approx(yt2, rel=1e-10)
    p2 = p1 * stats.norm.pdf(yt2, loc=y[1, 0], scale=np.sqrt(d2))
    p2 /= p2.sum()
    np.testing.assert_allclose(out["posterior"], p2, rtol=1e-8, atol=1e-300)


def test_posterior_learns_the_secret_with_many_releases(orc):
    rng = np.random.default_rng(4)
    G = 200
    y = rng.normal(0, 1, size=(G, 1, 64))
    hits = 0
    for seed in range(10):
        out = orc.finalize(y, [1.0], np.full(G, 100, np.uint64), np.full(G, FULL), seed, 0.05)
        assert abs(out["posterior"].sum() - 1.0) < 1e-12
        hits += int(np.argmax(out["posterior"]) == out["jstar"])
    assert hits >= 8    # total MI 200 * 0.05 = 10 nats: the secret leaks


def test_jstar_uniform(orc):
    y = np.zeros((1, 1, 64))
    js = [orc.finalize(y, [1.0], np.array([1], np.uint64), np.array([FULL]), s, 1.0)["jstar"]
          for s in range(6400)]
    counts = np.bincount(js, minlength=64)
    assert stats.chisquare(counts).pvalue > 1e-3


def test_null_probability_and_no_update(orc):
    # or_g with 48 worlds set: NULL with probability 16/64 (Sec. 3.2)
    orm = np.uint64((1 << 48) - 1)
    G = 20000
    y = np.ones((G, 1, 64))
    out = orc.finalize(y, [1.0], np.full(G, 10, np.uint64), np.full(G, orm), 3, 1.0, orc.INDEPENDENT)
    frac = out["is_null"].mean()
    assert abs(frac - 0.25) < 5 * np.sqrt(0.25 * 0.75 / G)
    assert np.all((out["flags"][out["is_null"] == 1] & orc.F_NULL) != 0)
    assert np.all(out["noised"][out["is_null"] == 1] == 0.0)
    # all worlds seen: never NULL
    out = orc.finalize(y[:500], [1.0], np.full(500, 10, np.uint64), np.full(500, FULL), 3, 1.0)
    assert out["is_null"].sum() == 0
    # a NULL release does not move the posterior
    out = orc.finalize(y[:1] * np.arange(64), [1.0], np.array([10], np.uint64),
                       np.array([np.uint64(1)]), 1, 1.0)
    if out["is_null"][0]:
        np.testing.assert_allclose(out["posterior"], np.full(64, 1 / 64), rtol=1e-14)


def test_unset_worlds_count_as_zero(orc):
    rng = np.random.default_rng(2)
    G = 50
    y = rng.normal(5, 2, size=(G, 2, 64))
    orm = np.array([np.uint64(rng.integers(1, 2**63)) | np.uint64(0xFFFF0000FFFF) for _ in range(G)])
    z = y.copy()
    for g in range(G):
        for j in range(64):
            if not (int(orm[g]) >> j) & 1:
                z[g, :, j] = 0.0
    a = orc.finalize(y, [2.0, 1.0], np.full(G, 100, np.uint64), orm, 5, 0.1)
    b = orc.finalize(z, [2.0, 1.0], np.full(G, 100, np.uint64), orm, 5, 0.1)
    for k in ("noised", "is_null", "flags", "posterior"):
        np.testing.assert_array_equal(a[k], b[k])


def test_zero_variance_and_diversity_flags(orc):
    y = np.full((3, 1, 64), 7.0)
    single_pu = np.uint64(0x00000000FFFFFFFF)        # one balanced PU: 32 worlds
    meta_n = np.array([100, 100, 10], np.uint64)
    meta_or = np.array([FULL, single_pu, single_pu])
    out = orc.finalize(y, [2.0], meta_n, meta_or, 0, 1.0, orc.INDEPENDENT)
    assert out["noised"][0] == 14.0 and out["flags"][0] & orc.F_ZEROVAR
    assert not out["flags"][0] & orc.F_DIVERSITY
    assert out["flags"][1] & orc.F_DIVERSITY          # >= 64 rows, 32 worlds
    assert not out["flags"][2] & orc.F_DIVERSITY      # too few rows to judge
