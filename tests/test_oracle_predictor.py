"""Pins of the oracle's reuse predictor (inputs, decision, labels, training):
closed forms, brute force and special cases that reduce to the depth rule."""
import numpy as np
import pytest

import gen
import oracle
from oracle import predictor as P
from oracle.cache import CacheSim, cached_derive, collect_samples


def random_theta(seed, scale=0.3):
    rs = np.random.default_rng(seed)
    return (rs.standard_normal(P.NPARAM) * scale).astype(np.float32)


def test_bf16_round_ties_to_even_and_matches_c_rounding():
    one = np.float32(1.0)
    cases = {1.0: 1.0, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6, 1 + 2 ** -8 + 2 ** -20: 1 + 2 ** -7,
             -(1 + 3 * 2 ** -8): -(1 + 2 ** -6), 3.0: 3.0}
    for x, want in cases.items():
        assert P.bf16_round(np.array([x], np.float32))[0] == np.float32(want), x
    rs = np.random.default_rng(0)
    xs = (rs.standard_normal(500) * 10 ** rs.uniform(-6, 6, 500)).astype(np.float32)
    got = P.bf16_round(xs)
    assert np.all(got.view(np.uint32) & 0xFFFF == 0)
    assert np.all(np.abs(got - xs) <= np.abs(xs) * 2.0 ** -8)
    ref = np.array([oracle.round_bf16(float(x)) for x in xs], np.float32)
    assert np.array_equal(got, ref)
    assert one == P.bf16_round(np.array([1.0], np.float32))[0]


def test_plog2_is_exact_at_powers_of_two_and_close_to_log2():
    x = np.float32(2.0) ** np.arange(-20, 21, dtype=np.float32)
    assert np.array_equal(P.plog2(x), np.arange(-20, 21, dtype=np.float32))
    assert P.plog2(np.array([3.0], np.float32))[0] == 1.5
    assert P.plog2(np.array([256.0], np.float32), 8)[0] == 0.0
    y = np.exp(np.random.default_rng(1).uniform(-5, 12, 10000)).astype(np.float32)
    err = P.plog2(y).astype(np.float64) - np.log2(y.astype(np.float64))
    # max of log2(m) - (m - 1) on [1, 2) is at m = 1 / ln 2
    bound = np.log2(1 / np.log(2)) - (1 / np.log(2) - 1)
    assert err.min() >= -bound - 1e-6 and err.max() <= 1e-6


def test_pinned_direction_is_the_unit_direction():
    rs = np.random.default_rng(2)
    pc = np.array([-600.123456789, -598.5, 37.25])
    pos = (pc[None, :] + rs.uniform(-300, 300, (2000, 3))).astype(np.float32)
    d, n = P.pinned_dir(pos, pc)
    ref = pos.astype(np.float64) - pc[None, :]
    nr = np.linalg.norm(ref, axis=1)
    assert np.allclose(n, nr, rtol=1e-6)
    assert np.abs(d - ref / nr[:, None]).max() < 1e-6
    assert np.abs(np.linalg.norm(d.astype(np.float64), axis=1) - 1).max() < 1e-6
    d0, _ = P.pinned_dir(pos, pc)
    assert np.array_equal(P.features(np.zeros((2000, 32)), d, d0, n)[:, 32:35], np.zeros((2000, 3), np.float32))


def test_pinned_logit_equals_float64_forward_within_rounding():
    rs = np.random.default_rng(3)
    th = random_theta(4)
    z = rs.standard_normal((3000, P.NZ)).astype(np.float32)
    l32 = P.logit_f32(z, th).astype(np.float64)
    _, _, l64 = P.forward64(th, z)
    assert np.abs(l32 - l64).max() < 1e-4 * (1 + np.abs(l64).max())
    far = np.abs(l64) > 1e-3
    assert np.array_equal(P.decide(z, th)[far], (1 / (1 + np.exp(-l64)) >= 0.5)[far])


def test_bce_closed_forms():
    assert abs(P.bce(np.zeros(4), np.array([0, 1, 0, 1])) - np.log(2)) < 1e-15
    l = np.array([3.0, -2.0, 40.0, -40.0])
    y = np.array([1, 1, 0, 0])
    want = np.mean([np.log1p(np.exp(-3.0)), np.log1p(np.exp(2.0)), 40.0 + np.log1p(np.exp(-40.0)),
                    np.log1p(np.exp(-40.0))])
    assert abs(P.bce(l, y) - want) < 1e-12


def test_backprop_matches_central_differences():
    """float64 backprop against central finite differences of the float64 loss
    (unrounded weights: the derivative is of the loss as a function of theta)."""
    rs = np.random.default_rng(5)
    th = rs.standard_normal(P.NPARAM) * 0.3
    Z = rs.standard_normal((64, P.NZ))
    y = (rs.uniform(size=64) < 0.4).astype(np.float64)
    _, g = P.grad64(th, Z, y, round_weights=False)
    idx = np.r_[rs.choice(P.NZ * P.NH, 60, replace=False), P.NZ * P.NH + np.arange(0, 128, 5), P.NPARAM - 1]
    h = 1e-6
    for i in idx:
        e = np.zeros(P.NPARAM)
        e[i] = h
        fd = (P.loss64(th + e, Z, y, False) - P.loss64(th - e, Z, y, False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_step_is_a_signed_step():
    """After one step m_hat = g and v_hat = g^2, so the update is lr g / (|g| + eps)."""
    g = np.array([0.5, -2e-3, 0.0, 7.0])
    th0 = np.array([1.0, 1.0, 1.0, 1.0])
    opt = P.Adam(4, lr=0.01)
    th1 = opt.step(th0, g)
    assert np.allclose(th1, th0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    th2 = opt.step(th1, g)  # constant gradient: the same step again
    assert np.allclose(th2 - th1, th1 - th0, atol=1e-12)


def test_training_separates_a_learnable_rule():
    rs = np.random.default_rng(6)
    Z = rs.standard_normal((4000, P.NZ)).astype(np.float32)
    y = ((Z[:, 32] ** 2 + Z[:, 33] ** 2) < 1.0).astype(np.float64)  # reuse iff small direction change
    th0 = gen.reuse_mlp_init(7)
    batches = [rs.permutation(4000)[i: i + 256] for _ in range(30) for i in range(0, 4000, 256)]
    th, losses = P.train64(th0, Z, y, batches, lr=3e-3)
    acc = np.mean(P.decide(Z, th.astype(np.float32)) == (y > 0))
    assert losses[-1] < 0.5 * losses[0] and acc > 0.95


def test_label_rule_cases():
    k = 10
    base = np.zeros((1, k, 11))
    base[..., 0] = 0.5
    base[..., 1:4] = 0.3
    base[0, 3, 0] = -0.2  # a Gaussian that is not kept

    def lab(mod):
        c = base.copy()
        mod(c)
        return bool(P.label(c, base)[0])

    assert lab(lambda c: None)
    assert lab(lambda c: c.__setitem__((0, 1, 0), 0.5 + 0.5 / 255))
    assert not lab(lambda c: c.__setitem__((0, 1, 0), 0.5 + 1.5 / 255))
    assert lab(lambda c: c.__setitem__((0, 2, 2), 0.3 + 0.9 / 255 / 0.5))      # colour x alpha within 1/255
    assert not lab(lambda c: c.__setitem__((0, 2, 2), 0.3 + 1.1 / 255 / 0.5))
    assert lab(lambda c: c.__setitem__((0, 3, 1), 0.9))                        # not kept: ignored
    assert not lab(lambda c: c.__setitem__((0, 3, 0), 0.1))                    # kept set differs
    assert lab(lambda c: c.__setitem__((0, 4, 5), 9.0))                        # scales are not compared


@pytest.fixture(scope="module")
def tiny_path():
    m = gen.tiny_scene()
    cams = []
    for f in range(12):
        ang = 0.01 * f
        R = np.array([[np.cos(ang), 0, -np.sin(ang)], [0, 1, 0], [np.sin(ang), 0, np.cos(ang)]])
        cams.append(gen.pinhole(R, np.array([0.1 * f, 0.0, -15.0]), 256, 256, 60.0))
    return m, cams


def test_learned_policy_reduces_to_always_and_never(tiny_path):
    """A predictor that always says reuse behaves like the depth rule held at
    D_max; one that never does decodes every visible anchor every frame."""
    m, cams = tiny_path
    always = np.zeros(P.NPARAM, np.float32)
    always[-1] = 1.0
    never = np.zeros(P.NPARAM, np.float32)
    never[-1] = -1.0
    sa, sd, sn = (CacheSim(m.n, 1500) for _ in range(3))
    reused = 0
    for cam in cams:
        ids_a, _, _, hit_a, line_a, _ = cached_derive(m, cam, sa, theta=always)
        sd.depth = sd.D
        ids_d, _, _, hit_d, line_d, _ = cached_derive(m, cam, sd)
        assert np.array_equal(hit_a, hit_d) and np.array_equal(line_a, line_d)
        _, _, _, hit_n, _, _ = cached_derive(m, cam, sn, theta=never)
        assert not hit_n.any()
        reused += int(hit_a.sum())
    assert reused > 0


def test_collected_samples_are_the_valid_lines(tiny_path):
    m, cams = tiny_path
    sim = CacheSim(m.n, 1500)
    cached_derive(m, cams[0], sim)
    for cam in cams[1:4]:
        vi, z, lab, margin = collect_samples(m, cam, sim)
        valid, line, _ = sim.peek(oracle.cull(m, cam))
        assert np.array_equal(vi, np.nonzero(valid)[0])
        ids = oracle.cull(m, cam)
        assert np.array_equal(z[:, :32], m.feat[ids[vi]])
        assert len(vi) > 0 and lab.dtype == bool and np.all(margin >= 0)
        cached_derive(m, cam, sim)
